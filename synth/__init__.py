"""Seeded synthetic wall-source quark propagators.

This module is the only code shared by the CPU oracle and the CUDA path: it
draws inputs and holds none of the correlator arithmetic.

Layout of one propagator time slice (the layout every consumer reads):
``S[site, row, col]`` complex, ``site = x + L*(y + L*z)``, ``row = alpha*3 + c``
(sink spin/colour), ``col = alpha'*3 + c'`` (source spin/colour of the wall
source).  A full field is ``S[t, site, 12, 12]``.

Distribution (the workload the paper measures on, a 16^3 x 32 lattice with a
wall source, Sec. 5, replaced by synthetic data): i.i.d. complex Gaussian
entries with Re, Im ~ N(0, 1/2) (so E|z|^2 = 1), each slice multiplied by
exp(-m_f * d), d = (t - t0) mod T.  The up and down quarks share one draw
(isospin limit, Sec. 4); the strange quark has its own stream.  An independent
down-quark stream exists for tests that need S_u != S_d.

Generator: SplitMix64 used as a counter-based generator.  For a key k and a
counter i the 64-bit output is mix(k + (i + 1) * 0x9E3779B97F4A7C15), with
mix() the SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014).  Two
uniforms per entry go through the Box-Muller transform in float64.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: stream ids: the light (u = d) quark, the strange quark, a separate d quark
STREAM_LIGHT, STREAM_STRANGE, STREAM_DOWN = 0, 1, 2


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _slice_key(seed: int, lattice: int, source: int, stream: int, t: int) -> np.uint64:
    with np.errstate(over="ignore"):
        tag = np.uint64((lattice << 40) | (source << 32) | (stream << 24) | t)
        k = _mix(np.array([np.uint64(seed) * GOLDEN], dtype=np.uint64))[0]
        return _mix(np.array([k ^ _mix(np.array([tag], dtype=np.uint64))[0]]))[0]


def gaussian_slice(V: int, key: np.uint64) -> np.ndarray:
    """One time slice of unit complex Gaussians, shape [V, 12, 12], complex128."""
    n = V * 144
    ctr = np.arange(2 * n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        bits = _mix(key + (ctr + np.uint64(1)) * GOLDEN)
    u = ((bits >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1)) * np.sqrt(0.5)
    ang = 2.0 * np.pi * u2
    return (rad * np.cos(ang) + 1j * rad * np.sin(ang)).reshape(V, 12, 12)


def time_distance(t: int, t0: int, T: int) -> int:
    """d = (t - t0) mod T, the distance used for the mass decay and normalisation."""
    return (t - t0) % T


def propagator(L: int, T: int, t0: int, mass: float, stream: int, seed: int = 0,
               lattice: int = 0, source: int = 0, times=None) -> np.ndarray:
    """Propagator field of one flavour stream, shape [len(times), L^3, 12, 12] complex128."""
    V = L ** 3
    times = range(T) if times is None else list(times)
    out = np.empty((len(times), V, 12, 12), dtype=np.complex128)
    for i, t in enumerate(times):
        key = _slice_key(seed, lattice, source, stream, t)
        out[i] = gaussian_slice(V, key) * np.exp(-mass * time_distance(t, t0, T))
    return out


def flavour_set(L: int, T: int, t0: int = 0, m_ud: float = 0.3, m_s: float = 0.4,
                seed: int = 0, lattice: int = 0, source: int = 0, times=None,
                isospin: bool = True) -> dict:
    """Propagators keyed by flavour 'u', 'd', 's'.

    With ``isospin`` the 'u' and 'd' entries are the same array object.
    """
    u = propagator(L, T, t0, m_ud, STREAM_LIGHT, seed, lattice, source, times)
    s = propagator(L, T, t0, m_s, STREAM_STRANGE, seed, lattice, source, times)
    d = u if isospin else propagator(L, T, t0, m_ud, STREAM_DOWN, seed, lattice, source, times)
    return {"u": u, "d": d, "s": s}


def plane_wave(L: int, P: np.ndarray, n: tuple) -> np.ndarray:
    """Colour-diagonal plane-wave propagator slice, shape [L^3, 12, 12].

    S[(a,c),(a',c')](x) = delta(c,c') P[a,a'] exp(i 2 pi n.x / L); used by the
    closed-form tests (the correlator of such inputs is known for every r).
    """
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    ph = np.exp(2j * np.pi * (n[0] * x + n[1] * y + n[2] * z) / L).reshape(-1)
    blk = np.kron(P, np.eye(3))
    return ph[:, None, None] * blk[None, :, :]
