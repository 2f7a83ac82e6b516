"""Write the oracle's correlators at sampled r for the full-size workloads.

Run from the repository root:  python tests/golden/make_oracle_goldens.py [case ...]

It imports only ``synth`` (the seeded inputs) and ``oracle`` (the CPU FP64
direct Wick enumeration), never the CUDA library, and writes one
``oracle_<case>.npz`` per case beside this file.  Each file holds the raw
correlator C_ch(r) of one time slice (Sec. 2 Eq. 2 without the normalisation
factor) at the listed relative distances r for the 52 channels of Sec. 4 (three of
them on the largest lattice),
plus what the GPU tests need to rebuild the same inputs: the lattice, the
generator tags, the storage type the propagators are rounded to, and a
checksum of the propagators (sum of |S|^2 per flavour) so that a test can
tell a changed generator from a wrong kernel.

The r samples are drawn from a seeded generator and always include r = 0 and
the points r = -r (mod L) where identical sink baryons give zero (Sec. 5
footnote); the oracle sums over every X for each sampled r.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
import oracle.oracle as orc  # noqa: E402

M_UD, M_S = 0.3, 0.4

#: name -> (L, T, t0, seed, lattice, source, slices, n_r, storage[, channels])
CASES = {
    # 16^3 x 32, one wall source, complex128 (the bench lattice of Sec. 5)
    "config2_L16_T32": (16, 32, 0, 0, 0, 0, [1, 8, 16, 31], 64, "c128"),
    # 32^3 x 64, slice t = T/2, complex128 (the precision comparison)
    "config3_L32_T64": (32, 64, 0, 3, 0, 0, [32], 65, "c128"),
    # two items of the uneven batch: complex64 storage, sources at t0 = T/4, T/2
    "config4_L24_T48": (24, 48, 12, 0, 3, 1, [20], 32, "c64"),
    "config4_L32_T64": (32, 64, 32, 0, 6, 2, [40], 16, "c64"),
    # 48^3 x 96, complex64 storage (the streamed lattice): three channels, as
    # the oracle's sink tensors of five baryons take 30 GB of host memory here
    "config5_L48_T96": (48, 96, 0, 0, 0, 0, [5], 8, "c64", [0, 10, 51]),
}


def r_samples(L: int, n: int, seed: int) -> np.ndarray:
    """r = 0, the other seven points with r = -r (mod L), then seeded distinct r."""
    h = L // 2
    special = [x + L * (y + L * z) for z in (0, h) for y in (0, h) for x in (0, h)]
    rng = np.random.default_rng(seed)
    rest = [int(v) for v in rng.permutation(L ** 3) if int(v) not in special]
    return np.array((special + rest)[:n], dtype=np.int32)


def inputs(L, T, t0, seed, lattice, source, t, storage):
    F = synth.flavour_set(L, T, t0, M_UD, M_S, seed=seed, lattice=lattice, source=source, times=[t])
    Su, Ss = F["u"][0], F["s"][0]
    if storage == "c64":  # the GPU reads complex64: the oracle sees the same rounded numbers
        Su = Su.astype(np.complex64).astype(np.complex128)
        Ss = Ss.astype(np.complex64).astype(np.complex128)
    return Su, Ss


def make(name: str) -> str:
    L, T, t0, seed, lattice, source, slices, n_r, storage = CASES[name][:9]
    chans = list(CASES[name][9]) if len(CASES[name]) > 9 else list(range(52))
    r = r_samples(L, n_r, seed=1510 + L)
    C = np.zeros((len(slices), len(chans), len(r), 16), dtype=np.complex128)
    chk = np.zeros((len(slices), 2))
    for i, t in enumerate(slices):
        t_start = time.time()
        Su, Ss = inputs(L, T, t0, seed, lattice, source, t, storage)
        chk[i] = [float(np.sum(np.abs(Su) ** 2)), float(np.sum(np.abs(Ss) ** 2))]
        C[i] = orc.correlator(L, Su, Su, Ss, chans, r_list=r)
        print(f"{name}: t={t} done in {time.time() - t_start:.0f} s", flush=True)
    path = os.path.join(HERE, f"oracle_{name}.npz")
    np.savez(path, L=L, T=T, t0=t0, seed=seed, lattice=lattice, source=source, slices=np.array(slices),
             r=r, channels=np.array(chans), storage=storage, m_ud=M_UD, m_s=M_S, C=C, checksum=chk)
    return path


if __name__ == "__main__":
    for n in (sys.argv[1:] or list(CASES)):
        print(make(n), flush=True)
