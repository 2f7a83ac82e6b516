"""Pins of the oracle's lower spin components (Sec. 5: the lower two Dirac
components of every external spinor index, antibaryons backward in time),
against the determinant brute force, the block structure of C gamma5 in the
Dirac representation, Grassmann antisymmetry and the plane-wave closed form."""
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


def run(L, S, chans, r=None, lower=True):
    return orc.correlator(L, S["u"], S["d"], S["s"], chans, r, lower=lower)


def close(a, b, tol=1e-12):
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() / scale < tol


@pytest.mark.parametrize("ch,spins", [
    (0, [(2, 3, 2, 3), (3, 3, 2, 3)]),      # p n <- p n
    (1, [(2, 3, 2, 3), (3, 2, 2, 2)]),      # p Lambda <- p Lambda
    (4, [(2, 3, 3, 2)]),                    # Sigma+ n <- p Lambda
    (16, [(3, 2, 2, 3)]),                   # p Xi- <- p Xi-
    (11, [(2, 3, 2, 3)]),                   # Lambda Lambda <- p Xi-
])
def test_lower_bruteforce_single_site(ch, spins):
    """L=1, S_u != S_d: lower components == the 6x6 determinant expansion with
    Dirac indices 2, 3 on all four external spinors."""
    S = one_slice(1, isospin=False, seed=21)
    B = bf.correlator(1, S, orc.channel_baryons(ch), spins, [0])[0]
    C = run(1, S, [ch])[0, 0, [sidx(*(x - 2 for x in s)) for s in spins]]
    assert close(C, B)


def test_lower_bruteforce_translation():
    S = one_slice(2, isospin=False, seed=22)
    ch, spins, rs = 5, [(3, 2, 2, 3)], [1, 6]
    B = bf.correlator(2, S, orc.channel_baryons(ch), spins, rs)[:, 0]
    C = run(2, S, [ch], rs)[0, :, sidx(1, 0, 0, 1)]
    assert close(C, B)


def test_lower_equals_upper_of_block_swapped_propagators():
    """In the Dirac representation C gamma5 = diag(J, J) is unchanged when the
    upper and lower spin blocks are swapped, so relabelling Dirac indices
    0 <-> 2, 1 <-> 3 on every propagator index maps lower components onto
    upper ones: C_lower(S) = C_upper(Pi S Pi)."""
    L = 2
    S = one_slice(L, isospin=False, seed=23)
    Pi = np.kron(np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]]), np.eye(3))
    Sp = {f: Pi @ S[f] @ Pi for f in "uds"}
    chans = [0, 1, 10, 16, 41, 51]
    assert close(run(L, S, chans), run(L, Sp, chans, lower=False))
    # and the lower components are not the upper ones
    assert not close(run(L, S, chans), run(L, S, chans, lower=False), 1e-3)


def test_lower_antisymmetry_identical_source():
    L = 2
    S = one_slice(L, isospin=True, seed=24)
    chans = [10, 14, 37]
    C = run(L, S, chans).reshape(len(chans), L ** 3, 2, 2, 2, 2)
    assert close(C, -C.swapaxes(2, 3))
    assert np.abs(C).max() > 0


def test_lower_plane_wave_closed_form():
    """Plane waves with 4x4 spin matrices that mix upper and lower components:
    C(r) = V delta(P1 + P2) e^{i P1.r} K, K the single-site lower value."""
    L = 4
    rng = np.random.default_rng(25)
    mom = {"u": (1, 0, 0), "d": (L - 1, 0, 0), "s": (0, 0, 0)}  # p n: total 3u+3d momenta cancel
    P = {f: rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4)) for f in "uds"}
    S = {f: synth.plane_wave(L, P[f], mom[f]) for f in "uds"}
    S1 = {f: np.kron(P[f], np.eye(3))[None] for f in "uds"}
    ch = 0  # p n <- p n: B1 = p = (u d u), P1 = 2 p_u + p_d
    C = run(L, S, [ch])[0]
    K = run(1, S1, [ch])[0, 0]
    V = L ** 3
    r = np.arange(V)
    x = r % L
    P1x = (2 * mom["u"][0] + mom["d"][0]) % L
    want = V * np.exp(2j * np.pi * P1x * x / L)[:, None] * K[None, :]
    assert np.abs(K).max() > 0
    assert close(C, want)
