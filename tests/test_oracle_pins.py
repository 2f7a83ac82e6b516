"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

Each test would fail on a plausible slip in the oracle: a wrong Wick sign or
index (brute force, antisymmetry), a wrong colour tensor (SU(3) invariance), a
wrong spin matrix (charge-conjugation identity, spin-rotation covariance), a
wrong position of B1 or sign of r (plane-wave closed form), wrong Lambda /
Sigma0 coefficients (isospin zeros), or a wrong quark content (Wick counts and
the paper's diagram counts).
"""
import math

import numpy as np
import pytest

import bruteforce as bf
import synth
import oracle.oracle as orc


def sidx(a, b, ap, bp):
    return a + 2 * (b + 2 * (ap + 2 * bp))


def one_slice(L, isospin, seed=0):
    F = synth.flavour_set(L, 1, seed=seed, isospin=isospin)
    return {k: v[0].copy() for k, v in F.items()}


def run(L, S, chans, r=None):
    return orc.correlator(L, S["u"], S["d"], S["s"], chans, r)


def close(a, b, tol=1e-12):
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() / scale < tol


def neg_site(r, L):
    x, y, z = r % L, (r // L) % L, r // (L * L)
    return (-x) % L + L * ((-y) % L + L * ((-z) % L))


# ---------------------------------------------------------------- spin basis
def test_charge_conjugation_matrix():
    """C gamma5 of the oracle: C = gamma4 gamma2 obeys C g_mu C^-1 = -g_mu^T
    (Sec. 2, below Eq. FieldOperator_N) in the Dirac representation with
    gamma4 = diag(1,1,-1,-1) (Sec. 5: upper components = positive parity)."""
    cg5 = orc.cg5()
    C = cg5 @ bf.GAMMA5  # gamma5^2 = 1
    Cinv = np.linalg.inv(C)
    for g in bf.GAMMA:
        assert np.allclose(C @ g @ Cinv, -g.T)
    assert np.allclose(bf.GAMMA[3], np.diag([1, 1, -1, -1]))
    assert np.allclose(cg5, -cg5.T)
    # C gamma5 does not mix upper and lower components
    assert np.allclose(cg5[:2, 2:], 0) and np.allclose(cg5[2:, :2], 0)


# ------------------------------------------------------------- brute force
BF_CASES = [
    (0, [(0, 1, 0, 1), (1, 1, 0, 1)]),      # p n <- p n
    (1, [(0, 1, 0, 1), (1, 0, 0, 0)]),      # p Lambda <- p Lambda
    (4, [(0, 1, 1, 0)]),                    # Sigma+ n <- p Lambda
    (16, [(1, 0, 0, 1)]),                   # p Xi- <- p Xi-
    (51, [(0, 1, 0, 1)]),                   # Xi- Xi0 <- Xi- Xi0
    (11, [(0, 1, 0, 1)]),                   # Lambda Lambda <- p Xi-
]


@pytest.mark.parametrize("ch,spins", BF_CASES)
def test_bruteforce_single_site(ch, spins):
    """L=1, S_u != S_d: oracle == full 6x6 determinant expansion (Sec. 3)."""
    S = one_slice(1, isospin=False, seed=3)
    B = bf.correlator(1, S, orc.channel_baryons(ch), spins, [0])[0]
    C = run(1, S, [ch])[0, 0, [sidx(*s) for s in spins]]
    assert close(C, B, 1e-12)


def test_bruteforce_translation():
    """L=2: B1 at X + r, B2 at X, sum over X (Sec. 3 Eq. for R(r))."""
    S = one_slice(2, isospin=False, seed=5)
    ch, spins, rs = 5, [(0, 1, 0, 1)], [1, 6]
    B = bf.correlator(2, S, orc.channel_baryons(ch), spins, rs)[:, 0]
    C = run(2, S, [ch], rs)[0, :, sidx(*spins[0])]
    assert close(C, B, 1e-12)


def test_wick_counts_and_paper_diagram_counts():
    """N_u! N_d! N_s! flavour-preserving Wick terms (Sec. 3 naive count), and
    the number of diagrams = that count / (identical-quark swaps inside each
    sink baryon) as listed in the paper's Tables (Sec. 4)."""
    content = {"p": "uud", "n": "udd", "Sigma+": "uus", "Sigma-": "dds", "Sigma0": "uds",
               "Lambda": "uds", "Xi0": "uss", "Xi-": "dss"}
    paper_diagrams = {0: 9, 1: 6, 2: 6, 3: 6, 4: 3, 5: 3, 6: 3, 7: 6, 8: 6, 9: 6,
                      10: 8, 11: 8, 12: 8, 13: 8, 14: 8, 15: 2, 16: 2, 17: 2, 18: 2, 19: 2, 20: 2,
                      27: 2, 33: 8, 38: 8, 41: 8, 42: 6, 43: 6, 45: 3, 46: 3, 48: 6, 51: 6}
    for ch in range(52):
        b = orc.channel_baryons(ch)
        q = "".join(content[x] for x in b[:2])
        want = math.prod(math.factorial(q.count(f)) for f in "uds")
        assert orc.wick_count(ch) == want
        swaps = 1
        for x in b[:2]:
            for f in "uds":
                swaps *= math.factorial(content[x].count(f))
        if ch in paper_diagrams:
            assert want // swaps == paper_diagrams[ch], (ch, b)


# ----------------------------------------------------- plane-wave closed form
@pytest.mark.parametrize("ch", [1, 5, 7, 0, 10])
def test_plane_wave_closed_form(ch):
    """Colour-diagonal plane waves S_f = delta_cc' P_f e^{i p_f.x}:
    C(r) = V delta(P1 + P2 = 0 mod 2pi/L) e^{i P1.r} K with K the single-site
    value (FFT identity of Sec. 3 Eq. LN.pLLp.FFT with one momentum mode)."""
    L = 4
    rng = np.random.default_rng(11)
    mom = {"u": (1, 0, 0), "d": (0, 1, 0), "s": (1, 2, 0)}
    P = {f: rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4)) for f in "uds"}
    S = {f: synth.plane_wave(L, P[f], mom[f]) for f in "uds"}
    S1 = {f: np.kron(P[f], np.eye(3))[None] for f in "uds"}
    content = {"p": "udu", "n": "udd", "Sigma+": "usu", "Sigma0": "dsu", "Lambda": "dsu"}
    b = orc.channel_baryons(ch)
    tot = np.zeros(3, int)
    P1 = np.zeros(3, int)
    for i, x in enumerate(b[:2]):
        for f in content[x]:
            tot += mom[f]
            if i == 0:
                P1 += mom[f]
    C = run(L, S, [ch])[0]
    K = run(1, S1, [ch])[0, 0]
    V = L ** 3
    if np.all(tot % L == 0):
        r = np.arange(V)
        x, y, z = r % L, (r // L) % L, r // (L * L)
        ph = np.exp(2j * np.pi * (P1[0] * x + P1[1] * y + P1[2] * z) / L)
        want = V * ph[:, None] * K[None, :]
        assert np.abs(K).max() > 0
        assert close(C, want, 1e-12)
        # the single-site factor itself against the determinant brute force
        sp = (0, 1, 0, 1)
        Kb = bf.correlator(1, S1, b, [sp], [0])[0, 0]
        assert abs(K[sidx(*sp)] - Kb) <= 1e-12 * np.abs(K).max()
    else:
        assert np.abs(C).max() <= 1e-12 * V * np.abs(K).max()


# ------------------------------------------------------------- invariances
def su3(rng):
    z = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    q, r = np.linalg.qr(z)
    q = q * (np.diag(r) / np.abs(np.diag(r)))
    return q / np.linalg.det(q) ** (1 / 3)


def su2(rng):
    a = rng.normal(size=4)
    a /= np.linalg.norm(a)
    return np.array([[a[0] + 1j * a[3], a[2] + 1j * a[1]], [-a[2] + 1j * a[1], a[0] - 1j * a[3]]])


CH_INV = [0, 1, 6, 10, 19, 38, 44, 51]


def test_sink_colour_gauge_invariance():
    """eps_abc is SU(3) invariant and each sink baryon sits on one site, so a
    random local SU(3) rotation of the sink colour changes no correlator."""
    L = 2
    S = one_slice(L, isospin=False, seed=7)
    rng = np.random.default_rng(1)
    G = np.stack([np.kron(np.eye(4), su3(rng)) for _ in range(L ** 3)])
    S2 = {f: np.einsum("xij,xjk->xik", G, S[f]) for f in "uds"}
    assert close(run(L, S2, CH_INV), run(L, S, CH_INV))


def test_source_colour_rotation_invariance():
    L = 2
    S = one_slice(L, isospin=False, seed=8)
    H = np.kron(np.eye(4), su3(np.random.default_rng(2)))
    S2 = {f: S[f] @ H for f in "uds"}
    assert close(run(L, S2, CH_INV), run(L, S, CH_INV))


def test_spin_rotation_covariance():
    """C gamma5 is a rotation scalar (W^T J W = det W J) and delta carries the
    external spin, so R = diag(W, W) on the sink (source) spin rotates the
    indices a, b (a', b') of C by W (by W^T on the right)."""
    L = 2
    S = one_slice(L, isospin=False, seed=9)
    rng = np.random.default_rng(3)
    W = su2(rng)
    R = np.kron(np.block([[W, np.zeros((2, 2))], [np.zeros((2, 2)), W]]), np.eye(3))
    C = run(L, S, CH_INV).reshape(len(CH_INV), -1, 2, 2, 2, 2)  # [..., b', a', b, a]
    Csink = run(L, {f: R @ S[f] for f in "uds"}, CH_INV).reshape(C.shape)
    want = np.einsum("ag,bd,crqpdg->crqpba", W, W, C)
    assert close(Csink, want)
    Csrc = run(L, {f: S[f] @ R for f in "uds"}, CH_INV).reshape(C.shape)
    want = np.einsum("gp,dq,crdgba->crqpba", W, W, C)
    assert close(Csrc, want)


def test_antisymmetry_identical_sink():
    """B1 = B2: the baryon fields anticommute, C_{ab}(r) = -C_{ba}(-r) (Sec. 5
    footnote: zero at a = b where r = -r mod L)."""
    L = 3
    S = one_slice(L, isospin=True, seed=4)
    chans = [10, 12, 33, 35]
    C = run(L, S, chans).reshape(len(chans), L ** 3, 2, 2, 2, 2)  # [c, r, b', a', b, a]
    neg = [neg_site(r, L) for r in range(L ** 3)]
    assert close(C, -C[:, neg].swapaxes(-1, -2))
    assert np.abs(C).max() > 0


def test_antisymmetry_identical_source():
    """Bbar3 = Bbar4 at one wall: C_{a'b'} = -C_{b'a'} (Sec. 5 footnote)."""
    L = 2
    S = one_slice(L, isospin=True, seed=6)
    chans = [10, 14, 15, 19, 21, 27, 33, 37]
    C = run(L, S, chans).reshape(len(chans), L ** 3, 2, 2, 2, 2)
    assert close(C, -C.swapaxes(2, 3))
    assert np.abs(C).max() > 0


def test_isospin_zero_channels():
    """The four channels the paper omits vanish when S_u = S_d (Sec. 4), and
    only then."""
    L = 2
    omitted = [52, 53, 54, 55]
    ref = np.abs(run(L, one_slice(L, True, 12), [10, 14, 41])).max()
    C = run(L, one_slice(L, True, 12), omitted)
    assert np.abs(C).max() <= 1e-13 * ref
    C2 = run(L, one_slice(L, False, 12), omitted)
    assert np.abs(C2).max() > 1e-3 * ref


def test_homogeneity():
    """C is a polynomial of degree n_l in S_light and n_s in S_strange."""
    L = 2
    S = one_slice(L, True, 13)
    lam, mu = 0.5, 2.0
    S2 = {"u": lam * S["u"], "d": lam * S["u"], "s": mu * S["s"]}
    chans = list(range(52))
    C, C2 = run(L, S, chans, [0, 3]), run(L, S2, chans, [0, 3])
    n_strange = {"p": 0, "n": 0, "Sigma+": 1, "Sigma-": 1, "Sigma0": 1, "Lambda": 1, "Xi0": 2, "Xi-": 2}
    for i, ch in enumerate(chans):
        ns = sum(n_strange[b] for b in orc.channel_baryons(ch)[:2])
        assert close(C2[i], C[i] * lam ** (6 - ns) * mu ** ns)
