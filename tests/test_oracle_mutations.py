"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of the oracle's C source (a sign of
C gamma5 or of the colour tensor, a Lambda or Sigma0 coefficient, the Wick
parity, the position of B1, a quark flavour, the sink spin, the Omega
phase), builds the copy with gcc, and checks that the mutant disagrees with
the numpy determinant brute force (Sec. 3) on at least one of a few fixed
cases.  The oracle under test is untouched; if its source changes so that a
mutation no longer applies, the case fails and must be brought up to date.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import bruteforce as bf
import synth
import oracle.oracle as orc

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "bbc_oracle.c")

MUTATIONS = {
    "lower block of C gamma5 negated": (
        "for (int j = 0; j < 4; j++) g_gam[0][i][j] = creal(cg5[i][j]);",
        "for (int j = 0; j < 4; j++) g_gam[0][i][j] = (i >= 2 ? -1 : 1) * creal(cg5[i][j]);"),
    "Lambda X_s coefficient -1/sqrt6": ("add_term(B_L, -2.0 * r6, 2, 0, 1);", "add_term(B_L, -1.0 * r6, 2, 0, 1);"),
    "Sigma0 X_d sign": ("add_term(B_S0, -r2, 1, 2, 0);", "add_term(B_S0, r2, 1, 2, 0);"),
    "Wick permutation parity dropped": ("sign[n] = (inv & 1) ? -1 : 1;", "sign[n] = 1;"),
    "B1 at X - r": ("int Xr = (x + rx) % L + L * ((y + ry) % L + L * ((z + rz) % L));",
                    "int Xr = (x - rx + L) % L + L * ((y - ry + L) % L + L * ((z - rz + L) % L));"),
    "one colour permutation with the wrong sign": ("static const double eps_s[6] = {1, 1, 1, -1, -1, -1};",
                                                   "static const double eps_s[6] = {1, 1, 1, -1, -1, 1};"),
    "Omega_z phase +i": ("const cplx eta[3] = {I, 1, -I};", "const cplx eta[3] = {I, 1, I};"),
    "Xi0 with a d quark": ('set_bar(B_X0, "Xi0", FL_U, FL_S, FL_S);', 'set_bar(B_X0, "Xi0", FL_D, FL_S, FL_S);'),
    "second sink spin reads the first": ("baryon_tensor(b, off + 1, T[1]);", "baryon_tensor(b, off, T[1]);"),
}

# (L, channel, spins (a, b, a', b'), sites r): a few decisive brute-force cases
CASES = [
    (1, 1, [(0, 1, 0, 1), (1, 0, 1, 1)], [0]),      # p Lambda <- p Lambda
    (1, 41, [(0, 1, 1, 0)], [0]),                   # a Sigma0 channel
    (1, 51, [(0, 1, 0, 1), (1, 1, 1, 0)], [0]),     # Xi- Xi0 <- Xi- Xi0
    (1, 0, [(0, 1, 0, 1), (1, 1, 0, 1)], [0]),      # p n <- p n
    (1, 90, [(0, 1, 1, 0)], [0]),                   # Omega_x Omega_z <- Omega_y Omega_z
    (3, 5, [(0, 1, 0, 1)], [1]),                    # translation (odd L: -r differs from r): B1 at X + r
]


def sidx(a, b, ap, bp):
    return a + 2 * (b + 2 * (ap + 2 * bp))


@pytest.fixture(scope="module")
def reference():
    out = []
    for L, ch, spins, rs in CASES:
        F = synth.flavour_set(L, 1, seed=101 + L, isospin=False)
        S = {k: v[0].copy() for k, v in F.items()}
        B = bf.correlator(L, S, orc.channel_baryons(ch), spins, rs)
        out.append((L, ch, spins, rs, S, B))
    return out


def _run(lib, L, S, ch, rs):
    V = L ** 3
    arrs = [np.ascontiguousarray(S[f], dtype=np.complex128).reshape(V, 12, 12) for f in "uds"]
    chans = np.array([ch], dtype=np.int32)
    r = np.array(rs, dtype=np.int32)
    out = np.zeros((1, len(rs), 16), dtype=np.complex128)
    rc = lib.oracle_correlator_components(L, arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data, 1,
                                          chans.ctypes.data, len(rs), r.ctypes.data, 0, out.ctypes.data)
    return out[0] if rc == 0 else None


def _build(tmp_path, text, name):
    src = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    src.write_text(text)
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-std=gnu11", "-o", str(so), str(src), "-lm"])
    lib = ctypes.CDLL(str(so))
    lib.oracle_correlator_components.restype = ctypes.c_int
    lib.oracle_correlator_components.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 3 + [
        ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    return lib


def _max_rel_err(lib, reference):
    worst = 0.0
    for L, ch, spins, rs, S, B in reference:
        C = _run(lib, L, S, ch, rs)
        if C is None:
            return np.inf  # the mutant refuses to run: caught
        got = C[:, [sidx(*s) for s in spins]]
        worst = max(worst, np.abs(got - B).max() / np.abs(B).max())
    return worst


def test_unmutated_copy_agrees(tmp_path, reference):
    lib = _build(tmp_path, open(SRC).read(), "orig")
    assert _max_rel_err(lib, reference) < 1e-12


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_mutation_is_caught(tmp_path, reference, name):
    text = open(SRC).read()
    a, b = MUTATIONS[name]
    assert text.count(a) == 1, f"mutation '{name}' no longer applies to the oracle source"
    lib = _build(tmp_path, text.replace(a, b), "mutant")
    assert _max_rel_err(lib, reference) > 1e-6, name
