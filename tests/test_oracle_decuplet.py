"""Pins of the oracle's decuplet channels (Sec. 4 footnote: the baryon operator
of Sec. 2 with Gamma1 = C gamma_l, Gamma2 = 1 and a spatial vector index l;
here the Omega-, taken with the phase eta_l = (i, 1, -i) that makes its
matrix real): Omega_l1 Omega_l2 <- Omega_l3 Omega_l4 (ids 64..144) and
p Omega_l <- p Omega_l' (ids 145..153).

A wrong Gamma1 (C gamma5 kept, a wrong l order or phase) breaks the vector
covariance under spin rotations; a wrong Wick sign or index breaks the
determinant brute force and the Grassmann antisymmetry; a wrong flavour
content breaks the Wick counts, the homogeneity and the factorisation of
p Omega into two three-quark determinants.
"""
import itertools

import numpy as np
import pytest

import bruteforce as bf
import synth
import oracle.oracle as orc

AX = "xyz"


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
    for l1, l2, l3, l4 in itertools.product(range(3), repeat=4):
        ch = orc.omega_channel(l1, l2, l3, l4)
        assert orc.channel_baryons(ch) == tuple("Omega_" + AX[l] for l in (l1, l2, l3, l4))
    for l, m in itertools.product(range(3), repeat=2):
        assert orc.channel_baryons(orc.p_omega_channel(l, m)) == ("p", "Omega_" + AX[l], "p", "Omega_" + AX[m])
    assert orc.channel_baryons(63) == ("n", "Sigma-", "n", "Sigma-")
    with pytest.raises(ValueError):
        orc.channel_baryons(406)


def test_vector_diquark_matrices():
    """eta_l C gamma_l is real, symmetric (C gamma_mu C^-1 = -gamma_mu^T with
    C^T = -C) and does not mix upper and lower components."""
    for l in range(3):
        g = orc.gamma(1 + l)
        want = bf.ETA[l] * bf.CMAT @ bf.GAMMA[l]
        assert np.allclose(want.imag, 0)
        assert np.array_equal(g, want.real)
        assert np.array_equal(g, g.T)
        assert not g[:2, 2:].any() and not g[2:, :2].any()
    assert np.array_equal(orc.gamma(0), orc.cg5())


def test_wick_counts():
    """Six identical strange quarks: 6! = 720 flavour-preserving terms; p Omega:
    2! 1! 3! = 12 (Sec. 3 naive count)."""
    for ch in (64, 100, 144):
        assert orc.wick_count(ch) == 720
    for ch in range(145, 154):
        assert orc.wick_count(ch) == 12


BF_CASES = [
    (orc.omega_channel(0, 0, 0, 0), [(0, 1, 0, 1), (1, 0, 0, 1)]),
    (orc.omega_channel(0, 1, 2, 1), [(0, 1, 1, 0), (1, 1, 0, 0)]),
    (orc.omega_channel(2, 2, 1, 0), [(0, 0, 1, 1), (1, 0, 1, 0)]),
    (orc.p_omega_channel(1, 2), [(0, 1, 0, 1), (1, 1, 0, 0)]),
]


@pytest.mark.parametrize("ch,spins", BF_CASES)
def test_bruteforce_single_site(ch, spins):
    """L = 1, S_u != S_d: oracle == full 6x6 determinant expansion (Sec. 3)."""
    S = one_slice(1, isospin=False, seed=61)
    B = bf.correlator(1, S, orc.channel_baryons(ch), spins, [0])[0]
    C = run(1, S, [ch])[0, 0, [sidx(*s) for s in spins]]
    assert close(C, B)
    assert np.abs(B).max() > 0


def test_bruteforce_translation():
    """L = 2: B1 at X + r, B2 at X, summed over X."""
    S = one_slice(2, isospin=False, seed=62)
    ch, spins, rs = orc.omega_channel(1, 0, 0, 1), [(0, 1, 1, 0)], [1, 6]
    B = bf.correlator(2, S, orc.channel_baryons(ch), spins, rs)[:, 0]
    C = run(2, S, [ch], rs)[0, :, sidx(*spins[0])]
    assert close(C, B)


def _so3(W):
    """R_lm with W^dagger sigma_l W = sum_m R_lm sigma_m (adjoint action of SU(2))."""
    s = bf._s
    return np.array([[0.5 * np.trace(s[m] @ W.conj().T @ s[l] @ W) for m in range(3)] for l in range(3)]).real


def _su2(rng):
    a = rng.normal(size=4)
    a /= np.linalg.norm(a)
    return np.array([[a[0] + 1j * a[3], a[2] + 1j * a[1]], [-a[2] + 1j * a[1], a[0] - 1j * a[3]]])


def _omega_tensor(L, S, fixed, sink):
    """C over the nine (l, l') of the sink pair (sink=True) or source pair with
    the other pair fixed: [3, 3, V, b', a', b, a]."""
    ids = []
    for l, m in itertools.product(range(3), repeat=2):
        ids.append(orc.omega_channel(l, m, *fixed) if sink else orc.omega_channel(*fixed, l, m))
    C = run(L, S, ids)
    return C.reshape(3, 3, L ** 3, 2, 2, 2, 2)


def test_vector_covariance():
    """A spin rotation diag(W, W) of the sink (source) indices turns eta_l C
    gamma_l into sum_m Rt_lm eta_m C gamma_m with Rt = eta R eta^-1 and R the
    rotation of W (W^T sigma2 sigma_l W = sum_m R_lm sigma2 sigma_m), and
    rotates the spins a, b (a', b') by W: the Omega_l operators transform as a
    vector times a spinor."""
    L = 2
    S = one_slice(L, isospin=True, seed=63)
    rng = np.random.default_rng(64)
    W = _su2(rng)
    eta = np.array(bf.ETA)
    Rot = np.kron(np.block([[W, np.zeros((2, 2))], [np.zeros((2, 2)), W]]), np.eye(3))
    # sink: the rotation acts on the propagator rows
    Rt = eta[:, None] * _so3(W) / eta[None, :]
    C = _omega_tensor(L, S, (0, 2), sink=True)
    Cr = _omega_tensor(L, {f: Rot @ S[f] for f in "uds"}, (0, 2), sink=True)
    want = np.einsum("lm,kn,ag,bd,mnrqpdg->lkrqpba", Rt, Rt, W, W, C)
    assert close(Cr, want)
    # source: on the columns, i.e. W^T on the source tensors
    Rs = eta[:, None] * _so3(W.T) / eta[None, :]
    C = _omega_tensor(L, S, (1, 1), sink=False)
    Cr = _omega_tensor(L, {f: S[f] @ Rot for f in "uds"}, (1, 1), sink=False)
    want = np.einsum("lm,kn,gp,dq,mnrdgba->lkrqpba", Rs, Rs, W, W, C)
    assert close(Cr, want)
    assert np.abs(C).max() > 0


def test_exchange_antisymmetry():
    """The baryon fields anticommute: exchanging the two sink operators gives
    C[l1 l2; a b](r) = -C[l2 l1; b a](-r); the two source operators at one
    wall, C[l3 l4; a' b'] = -C[l4 l3; b' a']."""
    L = 3
    S = one_slice(L, isospin=True, seed=65)
    pairs = [(0, 1, 2, 0), (2, 2, 0, 1), (1, 2, 1, 1)]
    neg = [neg_site(r, L) for r in range(L ** 3)]
    for l1, l2, l3, l4 in pairs:
        a = run(L, S, [orc.omega_channel(l1, l2, l3, l4)]).reshape(L ** 3, 2, 2, 2, 2)
        b = run(L, S, [orc.omega_channel(l2, l1, l3, l4)]).reshape(L ** 3, 2, 2, 2, 2)
        c = run(L, S, [orc.omega_channel(l1, l2, l4, l3)]).reshape(L ** 3, 2, 2, 2, 2)
        assert close(a, -b[neg].swapaxes(-1, -2))
        assert close(a, -c.swapaxes(1, 2))
        assert np.abs(a).max() > 0


def test_homogeneity():
    """Omega Omega is of degree 6 in S_strange and 0 in S_light; p Omega of
    degree 3 in each."""
    L = 2
    S = one_slice(L, True, 66)
    lam, mu = 0.5, 1.5
    S2 = {"u": lam * S["u"], "d": lam * S["u"], "s": mu * S["s"]}
    chans = [64, 101, 144, 145, 153]
    C, C2 = run(L, S, chans, [0, 5]), run(L, S2, chans, [0, 5])
    for i, ch in enumerate(chans):
        ns = 6 if ch < 145 else 3
        assert close(C2[i], C[i] * lam ** (6 - ns) * mu ** ns)


def _two_point(sink, src, S, ext_sink, ext_src):
    """Three-quark two-point function on one site, per site (sink and source
    operators of the same flavour string):
    sum T_sink(a; xi) T_src(a'; eta) det_{ij}[delta(f_i, f_j) S_{f_i}[xi_i, eta_j]]."""
    flav = bf.OPS[sink][0]
    assert bf.OPS[src][0] == flav
    e1, e3 = bf.tensor_entries(sink, ext_sink), bf.tensor_entries(src, ext_src)
    V = S["s"].shape[0]
    out = np.zeros(V, complex)
    for x in range(V):
        for k1, v1 in e1.items():
            for k3, v3 in e3.items():
                M = np.array([[S[flav[i]][x][k1[i], k3[j]] if flav[i] == flav[j] else 0.0 for j in range(3)]
                              for i in range(3)])
                out[x] += v1 * v3 * np.linalg.det(M)
    return out


def test_p_omega_factorises():
    """No quark is shared between p and Omega, so the 6x6 Wick determinant is
    block diagonal: C(r) = sum_X G_p(X + r)[a, a'] G_Omega(X)[b, b'] with G the
    three-quark two-point functions (a plain convolution of two baryon
    correlators)."""
    L = 2
    V = L ** 3
    S = one_slice(L, isospin=False, seed=67)
    for l, m in ((2, 0), (1, 1)):
        C = run(L, S, [orc.p_omega_channel(l, m)])[0]
        Gp = {(a, ap): _two_point("p", "p", S, a, ap) for a in range(2) for ap in range(2)}
        Go = {(b, bp): _two_point("Omega_" + AX[l], "Omega_" + AX[m], S, b, bp) for b in range(2) for bp in range(2)}
        want = np.zeros((V, 16), complex)
        for r in range(V):
            rx, ry, rz = r % L, (r // L) % L, r // (L * L)
            for X in range(V):
                x, y, z = X % L, (X // L) % L, X // (L * L)
                Xr = (x + rx) % L + L * ((y + ry) % L + L * ((z + rz) % L))
                for a, b, ap, bp in itertools.product(range(2), repeat=4):
                    want[r, sidx(a, b, ap, bp)] += Gp[(a, ap)][Xr] * Go[(b, bp)][X]
        assert close(C, want)
        assert np.abs(want).max() > 0


def test_plane_wave_closed_form():
    """Colour-diagonal plane waves of momentum p_s: C(r) = V e^{i P1.r} K when
    6 p_s = 0 mod L (P1 = 3 p_s, K the single-site value), zero otherwise."""
    rng = np.random.default_rng(68)
    P = {f: rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4)) for f in "uds"}
    ch = orc.omega_channel(0, 1, 1, 2)
    S1 = {f: np.kron(P[f], np.eye(3))[None] for f in "uds"}
    K = run(1, S1, [ch])[0, 0]
    assert np.abs(K).max() > 0
    for L, mom in ((6, (1, 2, 0)), (4, (1, 0, 1))):
        S = {f: synth.plane_wave(L, P[f], mom if f == "s" else (0, 0, 0)) for f in "uds"}
        rs = [0, 1, 7, L ** 3 - 1]
        C = run(L, S, [ch], rs)[0]
        V = L ** 3
        if all((6 * c) % L == 0 for c in mom):
            ph = [np.exp(2j * np.pi * sum(3 * c * v for c, v in zip(mom, (r % L, (r // L) % L, r // (L * L)))) / L)
                  for r in rs]
            want = V * np.array(ph)[:, None] * K[None, :]
            assert close(C, want)
        else:
            assert np.abs(C).max() <= 1e-12 * V * np.abs(K).max()


@pytest.mark.parametrize("ch,spins", [
    (orc.omega_channel(0, 2, 1, 1), [(2, 3, 2, 3), (3, 3, 3, 2)]),
    (orc.p_omega_channel(2, 0), [(2, 3, 3, 2)]),
])
def test_lower_components_bruteforce(ch, spins):
    """Lower Dirac components (Sec. 5) of decuplet channels: the determinant
    expansion with Dirac indices 2, 3 on all four external spinors."""
    S = one_slice(1, isospin=False, seed=69)
    B = bf.correlator(1, S, orc.channel_baryons(ch), spins, [0])[0]
    C = orc.correlator(1, S["u"], S["d"], S["s"], [ch], lower=True)[0, 0, [sidx(*(x - 2 for x in s)) for s in spins]]
    assert close(C, B)


def test_lower_equals_upper_of_block_swapped_propagators():
    """eta_l C gamma_l = diag(X, -X) changes sign when the upper and lower
    spin blocks are swapped, and every decuplet channel has an even number
    of Omega operators (C gamma5 of the proton is unchanged), so
    C_lower(S) = C_upper(Pi S Pi)."""
    L = 2
    S = one_slice(L, isospin=True, seed=70)
    Pi = np.kron(np.block([[np.zeros((2, 2)), np.eye(2)], [np.eye(2), np.zeros((2, 2))]]), np.eye(3))
    Sp = {f: Pi @ S[f] @ Pi for f in "uds"}
    chans = [64, 77, 130, 146, 152]
    lo = orc.correlator(L, S["u"], S["d"], S["s"], chans, lower=True)
    up = orc.correlator(L, Sp["u"], Sp["d"], Sp["s"], chans)
    assert close(lo, up)
    assert np.abs(lo).max() > 0
