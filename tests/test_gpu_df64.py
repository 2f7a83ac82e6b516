"""The FP64 path with double-float block-pair products (BBC_DF64) against the
FP64 oracle at the FP64 tolerance (GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
import oracle.oracle as orc

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1510_00903_gb300 import bbc  # noqa: E402

FP64_TOL = 1e-12


def _err(got, want):
    scale = np.abs(want).reshape(want.shape[0], -1).max(axis=1)
    return np.abs(got - want).reshape(want.shape[0], -1).max(axis=1) / scale


def test_df64_all_channels_L4():
    L, T, t = 4, 4, 3
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=91)
    ch = list(range(52)) + list(range(56, 64))
    cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=ch, precision=bbc.BBC_DF64, device=dev)
    got = cor.run(torch.from_numpy(F["u"][t:t + 1]).to(dev), torch.from_numpy(F["s"][t:t + 1]).to(dev), [t],
                  normalised=False)[0].cpu().numpy()
    want = orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], ch)
    e = _err(got, want)
    print(f"df64 L=4 all channels: max {e.max():.2e}")
    assert e.max() < FP64_TOL, e
    assert e.max() > 0  # really a different arithmetic from the FP64 path
    cor.close()


@pytest.mark.parametrize("L", [16, 24, 32])
def test_df64_sampled(L):
    T, t = 8, 5
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=92 + L, times=[t])
    ch = [0, 10, 41, 51]
    cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=ch, precision=bbc.BBC_DF64, device=dev)
    got = cor.run(torch.from_numpy(F["u"]).to(dev), torch.from_numpy(F["s"]).to(dev), [t],
                  normalised=False)[0].cpu().numpy()
    rs = [0, 1, L ** 3 // 3, L ** 3 - 1]
    want = orc.correlator(L, F["u"][0], F["d"][0], F["s"][0], ch, rs)
    scale = np.abs(want).reshape(len(ch), -1).max(axis=1)  # the oracle's scale
    err = np.abs(got[:, rs] - want).reshape(len(ch), -1).max(axis=1) / scale
    print(f"df64 L={L} sampled: max {err.max():.2e}")
    assert err.max() < FP64_TOL, err
    # against the plain FP64 path over every r
    cor64 = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=ch, precision=bbc.BBC_FP64, device=dev)
    ref = cor64.run(torch.from_numpy(F["u"]).to(dev), torch.from_numpy(F["s"]).to(dev), [t],
                    normalised=False)[0].cpu().numpy()
    e2 = _err(got, ref)
    print(f"df64 vs fp64 L={L}: max {e2.max():.2e}")
    assert e2.max() < FP64_TOL
    cor.close()
    cor64.close()
