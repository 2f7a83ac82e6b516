"""Python front end of the CPU FP64 oracle (``bbc_oracle.c``).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this module.  It never imports the CUDA
package and the CUDA package never imports it.

The oracle returns the raw correlator C_ch(r) of one time slice,
``out[channel, r, s]`` complex128, spin ``s = a + 2(b + 2(a' + 2 b'))`` over
the upper Dirac components; ``normalise`` multiplies by
exp((m_B1 + m_B2) d) as in Sec. 2 Eq. 2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bbc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libbbc_oracle.so")
_lib = None

BARYONS = ["p", "n", "Sigma+", "Sigma-", "Sigma0", "Lambda", "Xi0", "Xi-", "Omega_x", "Omega_y", "Omega_z",
           "Delta++_x", "Delta++_y", "Delta++_z", "Sigma*+_x", "Sigma*+_y", "Sigma*+_z", "Xi*0_x", "Xi*0_y", "Xi*0_z"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O3, OpenMP) into oracle/_build/."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-std=gnu11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_correlator.restype = ctypes.c_int
        L.oracle_correlator.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_correlator_components.restype = ctypes.c_int
        L.oracle_correlator_components.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                                   ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        L.oracle_channel_count.restype = ctypes.c_int
        L.oracle_threads.restype = ctypes.c_int
        L.oracle_channel_baryons.argtypes = [ctypes.c_int, ctypes.c_void_p]
        L.oracle_wick_count.argtypes = [ctypes.c_int]
        L.oracle_term_count.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.oracle_cg5.argtypes = [ctypes.c_void_p]
        L.oracle_gamma.argtypes = [ctypes.c_int, ctypes.c_void_p]
        L.oracle_gamma.restype = ctypes.c_int
        _lib = L
    return _lib


def threads() -> int:
    """OpenMP threads the oracle's loops over X run on."""
    return lib().oracle_threads()


def n_channels() -> int:
    """52 printed channels, the 4 omitted in the isospin limit, 8 other charge
    states, 81 Omega Omega and 9 p Omega channels."""
    return lib().oracle_channel_count()


def channel_baryons(ch: int) -> tuple:
    b = np.zeros(4, dtype=np.int32)
    if lib().oracle_channel_baryons(ch, b.ctypes.data) != 0:
        raise ValueError(f"bad channel {ch}")
    return tuple(BARYONS[i] for i in b)


def channel_name(ch: int) -> str:
    b = channel_baryons(ch)
    return f"{b[0]} {b[1]} <- {b[2]} {b[3]}"


def wick_count(ch: int) -> int:
    return lib().oracle_wick_count(ch)


def term_count(ch: int, ap: int, bp: int) -> int:
    return lib().oracle_term_count(ch, ap, bp)


def cg5() -> np.ndarray:
    out = np.zeros(16)
    lib().oracle_cg5(out.ctypes.data)
    return out.reshape(4, 4)


def gamma(g: int) -> np.ndarray:
    """Diquark matrix of the oracle's tensors: 0 = C gamma5, 1..3 = eta_l C gamma_l."""
    out = np.zeros(16)
    if lib().oracle_gamma(g, out.ctypes.data) != 0:
        raise ValueError(f"bad diquark matrix {g}")
    return out.reshape(4, 4)


def omega_channel(l1: int, l2: int, l3: int, l4: int) -> int:
    """Id of Omega_l1 Omega_l2 <- Omega_l3 Omega_l4 (l = 0, 1, 2 for x, y, z)."""
    return 64 + 27 * l1 + 9 * l2 + 3 * l3 + l4


def p_omega_channel(l: int, lp: int) -> int:
    """Id of p Omega_l <- p Omega_l'."""
    return 145 + 3 * l + lp


#: first id of the 81 vector combinations of each decuplet pair family
DECUPLET_PAIR_BASE = {"Omega": 64, "Delta++": 154, "Sigma*+": 235, "Xi*0": 316}


def decuplet_channel(family: str, l1: int, l2: int, l3: int, l4: int) -> int:
    """Id of D_l1 D_l2 <- D_l3 D_l4 for D in Omega, Delta++, Sigma*+, Xi*0."""
    return DECUPLET_PAIR_BASE[family] + 27 * l1 + 9 * l2 + 3 * l3 + l4


def p_delta_channel(l: int, lp: int) -> int:
    """Id of p Delta++_l <- p Delta++_l'."""
    return 397 + 3 * l + lp


def correlator(L: int, Su: np.ndarray, Sd: np.ndarray, Ss: np.ndarray, channels,
               r_list=None, lower: bool = False) -> np.ndarray:
    """Raw correlators of one time slice: [n_ch, n_r (or V), 16] complex128.

    Su, Sd, Ss: [V, 12, 12] complex128 propagator slices (sink row 3a+c,
    source column 3a'+c').  lower: the lower two Dirac components (2, 3) of
    every external spinor index instead of the upper two (Sec. 5), output
    spins relabelled to 0, 1.
    """
    V = L ** 3
    arrs = [np.ascontiguousarray(S, dtype=np.complex128).reshape(V, 12, 12) for S in (Su, Sd, Ss)]
    ch = np.ascontiguousarray(np.atleast_1d(channels), dtype=np.int32)
    if r_list is None:
        rl, nr, n_out = None, 0, V
    else:
        rl = np.ascontiguousarray(np.atleast_1d(r_list), dtype=np.int32)
        nr = n_out = len(rl)
    out = np.zeros((len(ch), n_out, 16), dtype=np.complex128)
    rc = lib().oracle_correlator_components(L, arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data,
                                            len(ch), ch.ctypes.data, nr,
                                            None if rl is None else rl.ctypes.data, int(bool(lower)),
                                            out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_correlator failed ({rc})")
    return out


#: synthetic hadron masses for the normalisation: the sum of the quark decay
#: masses of the generator (the paper divides by exp(-(m_B1 + m_B2)(t - t0))).
def baryon_mass(name: str, m_ud: float, m_s: float) -> float:
    n_s = {"p": 0, "n": 0, "Sigma+": 1, "Sigma-": 1, "Sigma0": 1, "Lambda": 1, "Xi0": 2, "Xi-": 2,
           "Omega_x": 3, "Omega_y": 3, "Omega_z": 3, "Delta++_x": 0, "Delta++_y": 0, "Delta++_z": 0,
           "Sigma*+_x": 1, "Sigma*+_y": 1, "Sigma*+_z": 1, "Xi*0_x": 2, "Xi*0_y": 2, "Xi*0_z": 2}[name]
    return (3 - n_s) * m_ud + n_s * m_s


def normalise(C: np.ndarray, channels, d: int, m_ud: float, m_s: float) -> np.ndarray:
    """R = C * exp((m_B1 + m_B2) d) per channel (Sec. 2 Eq. 2)."""
    out = np.array(C, copy=True)
    for i, ch in enumerate(np.atleast_1d(channels)):
        b = channel_baryons(int(ch))
        out[i] *= np.exp((baryon_mass(b[0], m_ud, m_s) + baryon_mass(b[1], m_ud, m_s)) * d)
    return out
