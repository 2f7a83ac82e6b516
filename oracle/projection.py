"""CPU FP64 oracle of the spin and cubic-group projections of Sec. 2.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this module.  It never imports the CUDA
package and the CUDA package never imports it.

Input is the correlator layout of the oracle (and of the library):
``C[..., site, s]`` with ``s = a + 2(b + 2(a' + 2 b'))`` over the upper Dirac
components (index 0 = spin up, 1 = spin down), ``site = x + L(y + L z)``.

* ``project_spin`` contracts the source spins (a', b') with the
  coefficients P^(J,M)_{a'b'} of the source operator of Sec. 2 (Eq. for
  R^(J,M)); the output index is ``j = a + 2 b + 4 jm`` over the states
  ``SPIN_STATES`` = (J,M) = (0,0), (1,+1), (1,0), (1,-1).
* ``project_a1`` is the operator P = (1/24) sum over the 24 rotations R of
  the cubic group O of R acting on the relative coordinate (Sec. 2, the
  3S1 / 3D1 split): (P f)(r) = (1/24) sum_R f(R^-1 r), the sink spin
  indices untouched.  Q = 1 - P gives the D-wave part.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

SPIN_STATES = [(0, 0), (1, 1), (1, 0), (1, -1)]


def spin_projector() -> np.ndarray:
    """P[jm, a', b']: the two-spin-1/2 state |J M> in the product basis
    |a'> x |b'> (Clebsch-Gordan coefficients, Condon-Shortley phases).
    Index 0 is m = +1/2, index 1 is m = -1/2."""
    h = 1.0 / math.sqrt(2.0)
    P = np.zeros((4, 2, 2))
    P[0, 0, 1], P[0, 1, 0] = h, -h      # J=0:        (|ud> - |du>)/sqrt2
    P[1, 0, 0] = 1.0                    # J=1, M=+1:  |uu>
    P[2, 0, 1], P[2, 1, 0] = h, h       # J=1, M=0:   (|ud> + |du>)/sqrt2
    P[3, 1, 1] = 1.0                    # J=1, M=-1:  |dd>
    return P


def project_spin(C: np.ndarray) -> np.ndarray:
    """R[..., a + 2b + 4jm] = sum_{a'b'} P[jm, a', b'] C[..., a + 2b + 4a' + 8b']."""
    C = np.asarray(C)
    P = spin_projector()
    Cs = C.reshape(C.shape[:-1] + (2, 2, 2, 2))          # [..., b', a', b, a]
    R = np.einsum("jpq,...qpba->...jba", P, Cs)           # p = a', q = b'
    return R.reshape(C.shape[:-1] + (16,))


def cubic_rotations() -> list:
    """The 24 proper rotations of the cube: the 3x3 signed permutation
    matrices with determinant +1."""
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            M = np.zeros((3, 3), dtype=np.int64)
            for i in range(3):
                M[i, perm[i]] = signs[i]
            if round(np.linalg.det(M)) == 1:
                mats.append(M)
    return mats


def project_a1(F: np.ndarray, L: int) -> np.ndarray:
    """(P F)[..., r, s] = (1/24) sum_R F[..., R^-1 r mod L, s] on the periodic
    L^3 lattice (integer rotations map the lattice onto itself)."""
    F = np.asarray(F)
    V = L ** 3
    idx = np.arange(V)
    r = np.stack([idx % L, (idx // L) % L, idx // (L * L)])   # [3, V]: x, y, z
    out = np.zeros(F.shape, dtype=np.result_type(F.dtype, np.float64))
    for M in cubic_rotations():
        src = (M.T @ r) % L                                    # R^-1 = R^T
        sidx = src[0] + L * (src[1] + L * src[2])
        out += np.take(F, sidx, axis=-2)
    return out / 24.0
