"""Pins of the oracle's other decuplet channels (Sec. 4 footnote: the baryon
operator of Sec. 2 with Gamma1 = C gamma_l, Gamma2 = 1): Delta++ Delta++,
Sigma*+ Sigma*+ and Xi*0 Xi*0 for all 81 vector-index combinations (ids
154..396) and p Delta++_l <- p Delta++_l' (ids 397..405).  The operators are a
reading (the footnote names the form and the Omega): Delta++ = eta_l eps
(u C gamma_l u) u, Sigma*+ = eta_l [eps (u C gamma_l u) s + 2 eps
(u C gamma_l s) u] / sqrt3, Xi*0 the same with u and s exchanged.

* Full 6 x 6 determinant brute force on one site with S_u != S_d (an
  independent evaluation of the Wick sum from the same operator definitions):
  catches a wrong sign, index or term of the two-term operators.
* Flavour relabelling: Delta++ is the Omega with u for s, Xi*0 the Sigma*+
  with u and s exchanged, so their correlators agree exactly once the
  propagators are exchanged the same way.
* Spin rotations: the operators transform as a vector times a spinor.
* Grassmann antisymmetry under exchange of the two sink or source operators.
* Homogeneity: the degree in S_light and S_strange of every channel.
"""
import itertools

import numpy as np
import pytest

import bruteforce as bf
import synth
import oracle.oracle as orc

AX = "xyz"
FAMILIES = {"Delta++": 0, "Sigma*+": 1, "Xi*0": 2}  # strange quarks per baryon


def sidx(a, b, ap, bp):
    return a + 2 * (b + 2 * (ap + 2 * bp))


def one_slice(L, isospin, seed=0):
    F = synth.flavour_set(L, 1, seed=seed, isospin=isospin)
    return {k: v[0].copy() for k, v in F.items()}


def run(L, S, chans, r=None):
    return orc.correlator(L, S["u"], S["d"], S["s"], chans, r)


def close(a, b, tol=1e-12):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300) < tol


def neg_site(r, L):
    x, y, z = r % L, (r // L) % L, r // (L * L)
    return (-x) % L + L * ((-y) % L + L * ((-z) % L))


def test_channel_table():
    assert orc.n_channels() == 406
    for fam in FAMILIES:
        for ls in itertools.product(range(3), repeat=4):
            ch = orc.decuplet_channel(fam, *ls)
            assert orc.channel_baryons(ch) == tuple(f"{fam}_{AX[l]}" for l in ls)
    assert [orc.decuplet_channel("Omega", *ls) for ls in itertools.product(range(3), repeat=4)] == \
        list(range(64, 145))
    for l, m in itertools.product(range(3), repeat=2):
        assert orc.channel_baryons(orc.p_delta_channel(l, m)) == ("p", "Delta++_" + AX[l], "p", "Delta++_" + AX[m])
    with pytest.raises(ValueError):
        orc.channel_baryons(406)


def test_wick_counts():
    """Delta++ Delta++: six u quarks, 6! = 720; Sigma*+ Sigma*+ and Xi*0 Xi*0:
    4! 2! = 48; p Delta++: five u and one d, 5! = 120."""
    for fam, n in (("Delta++", 720), ("Sigma*+", 48), ("Xi*0", 48)):
        for ls in ((0, 0, 0, 0), (1, 2, 0, 1), (2, 2, 2, 1)):
            assert orc.wick_count(orc.decuplet_channel(fam, *ls)) == n
    for ch in range(397, 406):
        assert orc.wick_count(ch) == 120


BF_CASES = [
    (orc.decuplet_channel("Delta++", 0, 1, 1, 0), [(0, 1, 0, 1), (1, 0, 1, 1)]),
    (orc.decuplet_channel("Sigma*+", 2, 1, 0, 2), [(0, 0, 1, 1), (1, 0, 1, 0)]),
    (orc.decuplet_channel("Xi*0", 0, 2, 1, 0), [(1, 0, 0, 0), (0, 1, 0, 1)]),
    (orc.p_delta_channel(1, 2), [(0, 1, 0, 1), (1, 1, 0, 0)]),
]


@pytest.mark.parametrize("ch,spins", BF_CASES)
def test_bruteforce_single_site(ch, spins):
    """L = 1, S_u != S_d: oracle == full 6x6 determinant expansion (Sec. 3)."""
    S = one_slice(1, isospin=False, seed=71)
    B = bf.correlator(1, S, orc.channel_baryons(ch), spins, [0])[0]
    C = run(1, S, [ch])[0, 0, [sidx(*s) for s in spins]]
    assert close(C, B)
    assert np.abs(B).max() > 0


def test_bruteforce_translation():
    """L = 2: B1 at X + r, B2 at X, summed over X."""
    S = one_slice(2, isospin=False, seed=72)
    ch, spins, rs = orc.decuplet_channel("Delta++", 1, 0, 0, 1), [(0, 1, 1, 0)], [1, 6]
    B = bf.correlator(2, S, orc.channel_baryons(ch), spins, rs)[:, 0]
    C = run(2, S, [ch], rs)[0, :, sidx(*spins[0])]
    assert close(C, B)


def test_flavour_relabelling():
    """Delta++ (u u u) is the Omega (s s s) with the flavour renamed, and Xi*0
    on (s, s, u) the Sigma*+ on (u, u, s) with u and s exchanged: exchanging
    the propagators the same way gives the same correlators (a spread of
    vector combinations)."""
    L = 2
    S = one_slice(L, isospin=True, seed=73)
    A, B = S["u"], S["s"]
    ls = list(itertools.product(range(3), repeat=4))[::10]
    ids = {f: [orc.decuplet_channel(f, *l) for l in ls] for f in ("Omega", "Delta++", "Sigma*+", "Xi*0")}
    de = orc.correlator(L, A, A, B, ids["Delta++"])  # S_u = A
    assert close(de, orc.correlator(L, B, B, A, ids["Omega"]))  # S_s = A
    assert not close(de, orc.correlator(L, A, A, B, ids["Omega"]))  # S_s = B: a different number
    sg = orc.correlator(L, A, A, B, ids["Sigma*+"])
    xi = orc.correlator(L, B, B, A, ids["Xi*0"])
    assert close(xi, sg)
    assert np.abs(sg).max() > 0


def _so3(W):
    s = bf._s
    return np.array([[0.5 * np.trace(s[m] @ W.conj().T @ s[l] @ W) for m in range(3)] for l in range(3)]).real


def _su2(rng):
    a = rng.normal(size=4)
    a /= np.linalg.norm(a)
    return np.array([[a[0] + 1j * a[3], a[2] + 1j * a[1]], [-a[2] + 1j * a[1], a[0] - 1j * a[3]]])


@pytest.mark.parametrize("fam", list(FAMILIES))
def test_vector_covariance(fam):
    """A spin rotation diag(W, W) of the sink indices turns eta_l C gamma_l into
    sum_m Rt_lm eta_m C gamma_m and rotates the spins a, b by W: each operator
    transforms as a vector times a spinor, both of its terms alike."""
    L = 2
    S = one_slice(L, isospin=True, seed=74)
    W = _su2(np.random.default_rng(75))
    eta = np.array(bf.ETA)
    Rot = np.kron(np.block([[W, np.zeros((2, 2))], [np.zeros((2, 2)), W]]), np.eye(3))
    Rt = eta[:, None] * _so3(W) / eta[None, :]

    def tensor(SS):
        ids = [orc.decuplet_channel(fam, l, m, 0, 2) for l, m in itertools.product(range(3), repeat=2)]
        return run(L, SS, ids).reshape(3, 3, L ** 3, 2, 2, 2, 2)

    C = tensor(S)
    Cr = tensor({f: Rot @ S[f] for f in "uds"})
    want = np.einsum("lm,kn,ag,bd,mnrqpdg->lkrqpba", Rt, Rt, W, W, C)
    assert close(Cr, want)
    assert np.abs(C).max() > 0


@pytest.mark.parametrize("fam", list(FAMILIES))
def test_exchange_antisymmetry(fam):
    """C[l1 l2; a b](r) = -C[l2 l1; b a](-r) (sink operators exchanged) and
    C[l3 l4; a' b'] = -C[l4 l3; b' a'] (source operators at one wall)."""
    L = 3
    S = one_slice(L, isospin=True, seed=76)
    neg = [neg_site(r, L) for r in range(L ** 3)]
    for l1, l2, l3, l4 in [(0, 1, 2, 0), (2, 2, 0, 1)]:
        a = run(L, S, [orc.decuplet_channel(fam, l1, l2, l3, l4)]).reshape(L ** 3, 2, 2, 2, 2)
        b = run(L, S, [orc.decuplet_channel(fam, l2, l1, l3, l4)]).reshape(L ** 3, 2, 2, 2, 2)
        c = run(L, S, [orc.decuplet_channel(fam, l1, l2, l4, l3)]).reshape(L ** 3, 2, 2, 2, 2)
        assert close(a, -b[neg].swapaxes(-1, -2))
        assert close(a, -c.swapaxes(1, 2))
        assert np.abs(a).max() > 0


def test_homogeneity():
    """Degree 6 - 2 n_s in S_light and 2 n_s in S_strange for the pairs of a
    baryon with n_s strange quarks; p Delta++ of degree 6 in S_light."""
    L = 2
    S = one_slice(L, True, 77)
    lam, mu = 0.5, 1.5
    S2 = {"u": lam * S["u"], "d": lam * S["u"], "s": mu * S["s"]}
    cases = [(orc.decuplet_channel(f, 1, 0, 2, 1), 2 * ns) for f, ns in FAMILIES.items()]
    cases.append((orc.p_delta_channel(0, 2), 0))
    chans = [c for c, _ in cases]
    C, C2 = run(L, S, chans, [0, 5]), run(L, S2, chans, [0, 5])
    for i, (ch, ns) in enumerate(cases):
        assert close(C2[i], C[i] * lam ** (6 - ns) * mu ** ns)
        assert np.abs(C[i]).max() > 0
