"""GPU parity of the decuplet channels (Sec. 4 footnote: Gamma1 = C gamma_l,
Gamma2 = 1): Omega_l1 Omega_l2 <- Omega_l3 Omega_l4 (ids 64..144) and
p Omega_l <- p Omega_l' (ids 145..153), through the C ABI against the oracle.

Tolerances as for the octet channels: FP64 and double-float 1e-12 of the
per-channel maximum; mixed (FP32 products, FP64 Wick sums) 2e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
import oracle.oracle as orc

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1510_00903_gb300 import bbc  # noqa: E402

FP64_TOL, MIXED_TOL = 1e-12, 2e-5
DECUPLET = list(range(64, 154))


def _err(got, want):
    scale = np.abs(want).reshape(want.shape[0], -1).max(axis=1)
    return np.abs(got - want).reshape(want.shape[0], -1).max(axis=1) / np.where(scale > 0, scale, 1.0)


def _run(L, T, t0, chans, F, t, precision=bbc.BBC_FP64, components=bbc.BBC_UPPER, normalised=False, k=None):
    """Slice t of the lattice; its propagators are F[...][k] (k = t unless given)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    cor = bbc.Correlators(L, T, t0, 0.3, 0.4, channels=chans, precision=precision, device=dev,
                          components=components)
    k = t if k is None else k
    Sl = torch.from_numpy(np.ascontiguousarray(F["u"][k:k + 1])).to(dev)
    Ss = torch.from_numpy(np.ascontiguousarray(F["s"][k:k + 1])).to(dev)
    out = cor.run(Sl, Ss, [t], normalised=normalised)[0].cpu().numpy()
    cor.close()
    return out


@pytest.fixture(scope="module")
def decuplet_L4():
    L, T, t = 4, 4, 2
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=91)
    want = orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], DECUPLET)
    return L, T, t, F, want


@pytest.mark.parametrize("precision,tol", [(bbc.BBC_FP64, FP64_TOL), (bbc.BBC_DF64, FP64_TOL),
                                           (bbc.BBC_MIXED_FP32, MIXED_TOL)])
def test_all_decuplet_channels_L4(decuplet_L4, precision, tol):
    """All 90 decuplet ids in one context, every r of one slice."""
    L, T, t, F, want = decuplet_L4
    got = _run(L, T, 0, DECUPLET, F, t, precision)
    e = _err(got, want)
    assert e.max() < tol, (e.max(), DECUPLET[int(e.argmax())])
    assert np.abs(want).reshape(len(DECUPLET), -1).max(axis=1).min() > 0


def test_mixed_unfused_route(decuplet_L4):
    """All 52 octet channels with the 90 decuplet ids exceed one CTA's shared
    memory in the fused kernel: mixed FP32 then runs the products and the
    Wick sums through a product buffer."""
    L, T, t, F, want_dec = decuplet_L4
    chans = list(range(52)) + DECUPLET
    want = np.concatenate([orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], list(range(52))), want_dec])
    got = _run(L, T, 0, chans, F, t, bbc.BBC_MIXED_FP32)
    e = _err(got, want)
    assert e.max() < MIXED_TOL, (e.max(), chans[int(e.argmax())])


def test_octet_and_decuplet_in_one_context():
    """Octet and decuplet families side by side in one block build (five
    diquarks per site), with the normalisation of each channel."""
    L, T, t0, t = 4, 6, 1, 4
    F = synth.flavour_set(L, T, t0, 0.3, 0.4, seed=92)
    chans = [0, 10, 41, 51, 60, 64, 98, 131, 144, 145, 153]
    got = _run(L, T, t0, chans, F, t, normalised=True)
    raw = orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], chans)
    e = _err(got, orc.normalise(raw, chans, t - t0, 0.3, 0.4))
    assert e.max() < FP64_TOL, e


def test_omega_L16_sampled():
    """L = 16 (the bench lattice), sampled r."""
    L, T, t = 16, 8, 3
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=93, times=[t])
    chans = [64, 76, 116, 144, 149]
    got = _run(L, T, 0, chans, F, t, k=0)
    rs = [0, 1, 17, 273, 2080, 4095]
    want = orc.correlator(L, F["u"][0], F["d"][0], F["s"][0], chans, rs)
    scale = np.abs(want).reshape(len(chans), -1).max(axis=1)  # the oracle's scale
    err = np.abs(got[:, rs] - want).reshape(len(chans), -1).max(axis=1) / scale
    assert err.max() < FP64_TOL, err


@pytest.mark.parametrize("precision,tol", [(bbc.BBC_FP64, FP64_TOL), (bbc.BBC_MIXED_FP32, MIXED_TOL)])
def test_omega_lower_components(precision, tol):
    """Lower Dirac components (Sec. 5) of the decuplet channels."""
    L, T, t0, t = 4, 6, 1, 4
    F = synth.flavour_set(L, T, t0, 0.3, 0.4, seed=94)
    chans = [64, 71, 100, 137, 146]
    got = _run(L, T, t0, chans, F, t, precision, components=bbc.BBC_LOWER)
    want = orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], chans, lower=True)
    e = _err(got, want)
    assert e.max() < tol, e
