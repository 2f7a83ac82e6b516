"""Pins of the oracle's other charge states (ids 56..63: pp, nn, S+S+, S-S-,
X0X0, X-X-, pS+, nS-) against the determinant brute force, the u <-> d
mirror of the isospin limit and the Grassmann antisymmetry of identical
baryons."""
import numpy as np
import pytest

import bruteforce as bf
import synth
import oracle.oracle as orc

OTHER = list(range(56, 64))


def sidx(a, b, ap, bp):
    return a + 2 * (b + 2 * (ap + 2 * bp))


def one_slice(L, isospin, seed=0):
    F = synth.flavour_set(L, 1, seed=seed, isospin=isospin)
    return {k: v[0].copy() for k, v in F.items()}


def run(L, S, chans, r=None):
    return orc.correlator(L, S["u"], S["d"], S["s"], chans, r)


def close(a, b, tol=1e-12):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300) < tol


def test_names():
    want = ["p p <- p p", "n n <- n n", "Sigma+ Sigma+ <- Sigma+ Sigma+", "Sigma- Sigma- <- Sigma- Sigma-",
            "Xi0 Xi0 <- Xi0 Xi0", "Xi- Xi- <- Xi- Xi-", "p Sigma+ <- p Sigma+", "n Sigma- <- n Sigma-"]
    assert orc.n_channels() == 406  # then the decuplet ids 64..405
    assert [orc.channel_name(c) for c in OTHER] == want


@pytest.mark.parametrize("ch", OTHER)
def test_bruteforce_single_site(ch):
    S = one_slice(1, isospin=False, seed=51)
    spins = [(0, 1, 0, 1), (1, 0, 0, 1), (1, 1, 1, 0)]
    B = bf.correlator(1, S, orc.channel_baryons(ch), spins, [0])[0]
    C = run(1, S, [ch])[0, 0, [sidx(*s) for s in spins]]
    assert close(C, B)


def test_isospin_mirror():
    """u <-> d maps p -> -n, Sigma+ -> Sigma-, Xi0 -> -Xi-: each channel and
    its mirror agree when the u and d propagators are exchanged."""
    L = 2
    S = one_slice(L, isospin=False, seed=52)
    Sm = {"u": S["d"], "d": S["u"], "s": S["s"]}
    for a, b in [(56, 57), (58, 59), (60, 61), (62, 63)]:
        assert close(run(L, S, [a]), run(L, Sm, [b]))
        assert not close(run(L, S, [a]), run(L, S, [b]), 1e-3)  # only through the exchange


def test_identical_baryon_antisymmetry():
    L = 3
    S = one_slice(L, isospin=True, seed=53)
    chans = list(range(56, 62))
    C = run(L, S, chans).reshape(len(chans), L ** 3, 2, 2, 2, 2)  # [c, r, b', a', b, a]
    assert close(C, -C.swapaxes(2, 3))  # identical source
    neg = [(-(r % L)) % L + L * ((-((r // L) % L)) % L + L * ((-(r // (L * L))) % L)) for r in range(L ** 3)]
    assert close(C, -C[:, neg].swapaxes(-1, -2))  # identical sink
