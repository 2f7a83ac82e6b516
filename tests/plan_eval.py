"""Host evaluation of a contraction plan (test infrastructure).

Runs the block algorithm of Sec. 3 in numpy, step by step, from the tables
`bbc_plan_export` returns: per-site sink-tensor families (diquark with
Gamma1 times a third propagator), block rows as weighted sums of their
entries, a forward FFT of every row (exp(-i q.x)), the block-pair products
A(q) B(-q) summed over the open index, the signed sums into channels and the
inverse FFT divided by V.  It shares no code with the CUDA kernels: the gamma
matrices come from `bruteforce` (numpy, from their definitions) and every
step is a plain numpy expression, so agreement with the oracle checks the
planner's tables on any lattice size, without a GPU.
"""
from __future__ import annotations

import itertools

import numpy as np

import bruteforce as bf

# (flavour of diquark quark 0, of diquark quark 1, of the third quark) with
# 0 = light, 1 = strange, and the diquark matrix Gamma1 of families 0..21:
# the four C gamma5 families, then (s s s) with eta_l C gamma_l (l = x, y, z),
# then, l = x, y, z each, (l l l), (l l s), (l s l), (l s s), (s s l) with
# eta_l C gamma_l (the family order of the plan's tensor indices)
_EPS = np.zeros((3, 3, 3))
for _p in itertools.permutations(range(3)):
    _EPS[_p] = 1.0 if sum(_p[i] > _p[j] for i in range(3) for j in range(i + 1, 3)) % 2 == 0 else -1.0
FAMILIES = [((0, 0, 0), bf.CG5), ((0, 0, 1), bf.CG5), ((0, 1, 0), bf.CG5), ((0, 1, 1), bf.CG5),
            ((1, 1, 1), bf.CGL[0]), ((1, 1, 1), bf.CGL[1]), ((1, 1, 1), bf.CGL[2])]
for _fl in ((0, 0, 0), (0, 0, 1), (0, 1, 0), (0, 1, 1), (1, 1, 0)):
    FAMILIES += [(_fl, bf.CGL[_l]) for _l in range(3)]


def family_tensors(S_light: np.ndarray, S_strange: np.ndarray, spin_offset: int) -> np.ndarray:
    """F[family][site][a*1728 + e0*144 + e1*12 + e2] =
    sum eps(c0,c1,c2) Gamma1(a0,a1) S_f0[(a0,c0),e0] S_f1[(a1,c1),e1] S_f2[(a+o,c2),e2]."""
    V = S_light.shape[0]
    S = [S_light.reshape(V, 4, 3, 12), S_strange.reshape(V, 4, 3, 12)]
    out = np.zeros((len(FAMILIES), V, 2 * 1728), complex)
    for f, ((f0, f1, f2), G) in enumerate(FAMILIES):
        assert np.allclose(G.imag, 0)
        D = np.einsum("ab,ijk,xaie,xbjf->xefk", G.real, _EPS, S[f0], S[f1])          # [V, e0, e1, c2]
        T = S[f2][:, spin_offset:spin_offset + 2]                                  # [V, a, c2, e2]
        out[f] = np.einsum("xefk,xakg->xaefg", D, T).reshape(V, -1)
    return out


def correlator(plan: dict, L: int, S_light: np.ndarray, S_strange: np.ndarray, spin_offset: int = 0) -> np.ndarray:
    """Raw correlators [n_channels, V, 16] of one slice from the plan tables."""
    V = L ** 3
    F = family_tensors(S_light, S_strange, spin_offset)
    row_ptr, terms = plan["row_ptr"], plan["terms"]
    n_out = len(row_ptr) - 1
    row_of_term = np.repeat(np.arange(n_out), np.diff(row_ptr))
    vals = F[terms[:, 0], :, terms[:, 1]] * terms[:, 2][:, None]                  # [n_terms, V]
    rows = np.zeros((n_out, V), complex)
    np.add.at(rows, row_of_term, vals)
    # sites x + L (y + L z): axes (z, y, x) after the reshape
    Ft = np.fft.fftn(rows.reshape(n_out, L, L, L), axes=(1, 2, 3)).reshape(n_out, V)
    q = np.arange(V)
    qx, qy, qz = q % L, (q // L) % L, q // (L * L)
    neg = (-qx) % L + L * ((-qy) % L + L * ((-qz) % L))
    tasks = plan["tasks"]
    P = np.zeros((16 * len(tasks), V), complex)
    for t, k in enumerate(tasks):
        nA, nB, n1, n2, sA1, sA2, sB1, sB2 = (int(x) for x in k[:8])
        i1, i2 = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
        for rA in range(nA):
            A = Ft[k[8 + rA] + i1.ravel() * sA1 + i2.ravel() * sA2]                   # [K, V] at q
            for rB in range(nB):
                B = Ft[k[16 + rB] + i1.ravel() * sB1 + i2.ravel() * sB2][:, neg]      # [K, V] at -q
                P[16 * t + rA * nB + rB] = (A * B).sum(axis=0)
    out_ptr, items, coefs = plan["out_ptr"], plan["items"], plan["coefs"]
    n_outputs = len(out_ptr) - 1
    Ct = np.zeros((n_outputs, V), complex)
    for o in range(n_outputs):
        sl = slice(out_ptr[o], out_ptr[o + 1])
        Ct[o] = (coefs[sl][:, None] * P[items[sl]]).sum(axis=0)
    C = np.fft.ifftn(Ct.reshape(n_outputs, L, L, L), axes=(1, 2, 3)).reshape(n_outputs, V)
    return C.reshape(n_outputs // 16, 16, V).transpose(0, 2, 1)
