"""Parity of the lower spin components (Sec. 5) with the oracle (GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
import oracle.oracle as orc

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1510_00903_gb300 import bbc  # noqa: E402

FP64_TOL, MIXED_TOL = 1e-12, 2e-5


def _err(got, want):
    scale = np.abs(want).reshape(want.shape[0], -1).max(axis=1)
    return np.abs(got - want).reshape(want.shape[0], -1).max(axis=1) / scale


@pytest.mark.parametrize("precision,tol", [(bbc.BBC_FP64, FP64_TOL), (bbc.BBC_MIXED_FP32, MIXED_TOL)])
def test_lower_all_channels_L4(precision, tol):
    L, T, t0, t = 4, 6, 1, 4
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, t0, 0.3, 0.4, seed=41)
    ch = list(range(52))
    cor = bbc.Correlators(L, T, t0, 0.3, 0.4, channels=ch, precision=precision, device=dev,
                          components=bbc.BBC_LOWER)
    Sl, Ss = torch.from_numpy(F["u"][t:t + 1]).to(dev), torch.from_numpy(F["s"][t:t + 1]).to(dev)
    got = cor.run(Sl, Ss, [t], normalised=True)[0].cpu().numpy()
    raw = orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], ch, lower=True)
    want = orc.normalise(raw, ch, (t0 - t) % T, 0.3, 0.4)  # backward time distance
    e = _err(got, want)
    assert e.max() < tol, e
    cor.close()


def test_lower_sampled_L16():
    L, T, t = 16, 8, 3
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=42, times=[t])
    ch = [0, 10, 41, 51]
    cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=ch, device=dev, components=bbc.BBC_LOWER)
    got = cor.run(torch.from_numpy(F["u"]).to(dev), torch.from_numpy(F["s"]).to(dev), [t],
                  normalised=False)[0].cpu().numpy()
    rs = [0, 1, 777, 4095]
    want = orc.correlator(L, F["u"][0], F["d"][0], F["s"][0], ch, rs, lower=True)
    scale = np.abs(want).reshape(len(ch), -1).max(axis=1)  # the oracle's scale
    err = np.abs(got[:, rs] - want).reshape(len(ch), -1).max(axis=1) / scale
    assert err.max() < FP64_TOL, err
    cor.close()
