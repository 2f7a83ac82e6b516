"""Brute-force Wick contraction with numpy determinants (an oracle pin).

Independent of the oracle's C code: the six-quark matrix element is evaluated
as a full 6x6 determinant (LU through numpy.linalg.det, zero blocks between
flavours included) for every pair of non-zero sink and source tensor entries:

  C_{a b a' b'}(r) = sum_X sum_{xi, eta} T_B1(a; xi1..3) T_B2(b; xi4..6)
                     T_B3(a'; eta1..3) T_B4(b'; eta4..6) det M(xi, eta),
  M_ij = delta(f_i, g_j) S_{f_i}(x_i)[xi_i, eta_j],

x_1..3 = X + r, x_4..6 = X (Sec. 3 Eq. for the p-Lambda correlator and the
Wick expansion after it, which is this determinant written out).  The
operators are the paper's Sec. 2 definitions (p, n: Eq. FieldOperator_N;
Sigma, Lambda, Xi, X_q: Eqs. FieldOperator_SLXi and FieldOperator_xxx) and
the decuplet of the Sec. 4 footnote (Gamma1 = C gamma_l, Gamma2 = 1): Omega-,
Delta++ and the flavour-symmetric Sigma*+, Xi*0, taken with the phase
eta_l = (i, 1, -i) that makes the matrix real.
Cost grows as (#sink entries) x (#source entries) x V: tiny lattices only.
"""
from __future__ import annotations

import itertools

import numpy as np

# gamma matrices (Dirac representation) and C gamma5, C = gamma4 gamma2
_s = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]]),
      np.array([[1, 0], [0, -1]], complex)]
_Z = np.zeros((2, 2))
GAMMA = [np.block([[_Z, -1j * s], [1j * s, _Z]]) for s in _s] + [np.diag([1, 1, -1, -1]).astype(complex)]
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
CMAT = GAMMA[3] @ GAMMA[1]
CG5 = CMAT @ GAMMA5
ETA = [1j, 1.0, -1j]
CGL = [ETA[l] * CMAT @ GAMMA[l] for l in range(3)]  # eta_l C gamma_l, l = x, y, z

r6, r2 = 1 / np.sqrt(6), 1 / np.sqrt(2)
# name -> (string flavours, [(coef, gamma slot i, gamma slot j, delta slot k)])
OPS = {
    "p": ("udu", [(1.0, 0, 1, 2)]),
    "n": ("udd", [(-1.0, 0, 1, 2)]),
    "Sigma+": ("usu", [(-1.0, 0, 1, 2)]),
    "Sigma-": ("dsd", [(-1.0, 0, 1, 2)]),
    "Xi0": ("uss", [(1.0, 0, 1, 2)]),
    "Xi-": ("dss", [(-1.0, 0, 1, 2)]),
    "Lambda": ("dsu", [(r6, 0, 1, 2), (r6, 1, 2, 0), (-2 * r6, 2, 0, 1)]),
    "Sigma0": ("dsu", [(r2, 0, 1, 2), (-r2, 1, 2, 0)]),
    "Omega_x": ("sss", [(1.0, 0, 1, 2)]),
    "Omega_y": ("sss", [(1.0, 0, 1, 2)]),
    "Omega_z": ("sss", [(1.0, 0, 1, 2)]),
}
# the other decuplet baryons in the same form (flavour-symmetric combinations):
# Delta++ = eps (u G u) u; Sigma*+ = [eps (u G u) s + 2 eps (u G s) u] / sqrt3 on
# the string (u, u, s); Xi*0 the same on (s, s, u)
_r3 = 1 / np.sqrt(3)
for _l, _ax in enumerate("xyz"):
    OPS["Delta++_" + _ax] = ("uuu", [(1.0, 0, 1, 2)])
    OPS["Sigma*+_" + _ax] = ("uus", [(_r3, 0, 1, 2), (2 * _r3, 0, 2, 1)])
    OPS["Xi*0_" + _ax] = ("ssu", [(_r3, 0, 1, 2), (2 * _r3, 0, 2, 1)])
# diquark matrix Gamma1 of each operator (C gamma5 unless listed)
GAM = {}
for _l, _ax in enumerate("xyz"):
    for _b in ("Omega_", "Delta++_", "Sigma*+_", "Xi*0_"):
        GAM[_b + _ax] = CGL[_l]


def _eps():
    out = []
    for p in itertools.permutations(range(3)):
        inv = sum(1 for i in range(3) for j in range(i + 1, 3) if p[i] > p[j])
        out.append((p, -1.0 if inv % 2 else 1.0))
    return out


def tensor_entries(name: str, ext: int):
    """Non-zero entries {(q0, q1, q2): value} of the baryon tensor, q = 3*spin + colour."""
    flav, terms = OPS[name]
    gam = GAM.get(name, CG5)
    assert np.allclose(gam.imag, 0)
    ent = {}
    for coef, i, j, k in terms:
        for cols, es in _eps():
            for ai in range(4):
                for aj in range(4):
                    g = gam[ai, aj].real
                    if g == 0:
                        continue
                    sp = [0, 0, 0]
                    sp[i], sp[j], sp[k] = ai, aj, ext
                    key = tuple(3 * sp[m] + cols[m] for m in range(3))
                    ent[key] = ent.get(key, 0.0) + coef * es * g
    return {k: v for k, v in ent.items() if v != 0.0}


def correlator(L: int, S: dict, chan: tuple, spins, r_sites) -> np.ndarray:
    """C for a channel (B1, B2, B3, B4), spin tuples (a, b, a', b'), sites r.

    S: flavour -> [V, 12, 12] propagator slice.  Returns [len(r_sites), len(spins)].
    """
    B1, B2, B3, B4 = chan
    V = L ** 3
    fs = OPS[B1][0] + OPS[B2][0]
    fg = OPS[B3][0] + OPS[B4][0]
    mask = np.array([[1.0 if fs[i] == fg[j] else 0.0 for j in range(6)] for i in range(6)])
    out = np.zeros((len(r_sites), len(spins)), complex)

    def coords(s):
        return s % L, (s // L) % L, s // (L * L)

    for si, (a, b, ap, bp) in enumerate(spins):
        e1, e2 = tensor_entries(B1, a), tensor_entries(B2, b)
        e3, e4 = tensor_entries(B3, ap), tensor_entries(B4, bp)
        sink = [(k1 + k2, v1 * v2) for k1, v1 in e1.items() for k2, v2 in e2.items()]
        src = [(k3 + k4, v3 * v4) for k3, v3 in e3.items() for k4, v4 in e4.items()]
        xi = np.array([k for k, _ in sink])            # [n_sink, 6]
        wx = np.array([v for _, v in sink])
        eta = np.array([k for k, _ in src])            # [n_src, 6]
        we = np.array([v for _, v in src])
        for ri, r in enumerate(r_sites):
            rx, ry, rz = coords(r)
            acc = 0.0 + 0.0j
            for X in range(V):
                x, y, z = coords(X)
                Xr = (x + rx) % L + L * ((y + ry) % L + L * ((z + rz) % L))
                site = [Xr, Xr, Xr, X, X, X]
                # P[i][row, col] = S_{f_i}(x_i)[row, col]
                P = np.stack([S[fs[i]][site[i]] for i in range(6)])  # [6, 12, 12]
                for c0 in range(0, len(sink), 256):
                    xs = xi[c0:c0 + 256]
                    # M[n_sink_chunk, n_src, i, j] = mask_ij * P_i[xi_i, eta_j]
                    rows = P[np.arange(6)[None, :], xs]             # [nc, 6, 12]
                    M = np.empty((len(xs), len(eta), 6, 6), complex)
                    for i in range(6):
                        for j in range(6):
                            if mask[i, j]:
                                M[:, :, i, j] = rows[:, i, :][:, eta[:, j]]
                            else:
                                M[:, :, i, j] = 0.0
                    d = np.linalg.det(M)                             # [nc, n_src]
                    acc += wx[c0:c0 + 256] @ d @ we
            out[ri, si] = acc
    return out
