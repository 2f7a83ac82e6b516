"""Edge cases of the GPU path: an empty slice list, zero propagators, and
propagators far outside the FP32 range (the exact power-of-two rescaling of
the ingest keeps the mixed path finite and correct), odd T and slot counts
that do not divide the slice list (GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
import oracle.oracle as orc

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1510_00903_gb300 import bbc  # noqa: E402


def _err(got, want):
    scale = np.abs(want).reshape(want.shape[0], -1).max(axis=1)
    return np.abs(got - want).reshape(want.shape[0], -1).max(axis=1) / scale


def test_empty_slice_list():
    dev = torch.device("cuda", torch.cuda.current_device())
    cor = bbc.Correlators(4, 4, 0, 0.3, 0.4, channels=[0, 1], device=dev)
    S = torch.zeros((0, 64, 12, 12), dtype=torch.complex128, device=dev)
    out = cor.run(S, S, [])
    assert tuple(out.shape) == (0, 2, 64, 16)
    cor.close()


@pytest.mark.parametrize("precision", [bbc.BBC_FP64, bbc.BBC_MIXED_FP32])
def test_zero_propagators_give_zero(precision):
    dev = torch.device("cuda", torch.cuda.current_device())
    cor = bbc.Correlators(4, 4, 0, 0.3, 0.4, channels=[0, 10, 51], precision=precision, device=dev)
    bbc.bbc_set_checks(cor.ctx, bbc.BBC_CHECK_INPUT | bbc.BBC_CHECK_OUTPUT)
    S = torch.zeros((1, 64, 12, 12), dtype=torch.complex128, device=dev)
    out = cor.run(S, S, [2]).cpu().numpy()
    assert np.all(out == 0)
    cor.close()


@pytest.mark.parametrize("e", [100, -100])
def test_mixed_path_outside_fp32_range(e):
    """S x 2^e with |e| = 100: C scales by 2^(6e) (six propagators), within
    FP64 but far outside FP32 (products of FP32 values would overflow or
    underflow).  The mixed path rescales each propagator by an exact power of
    two and undoes it in FP64."""
    L, T, t = 4, 4, 1
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=81, times=[t])
    ch = [0, 10, 41, 51]
    f = 2.0 ** e
    cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=ch, precision=bbc.BBC_MIXED_FP32, device=dev)
    Sl = torch.from_numpy(F["u"] * f).to(dev)
    Ss = torch.from_numpy(F["s"] * f).to(dev)
    got = cor.run(Sl, Ss, [t], normalised=False)[0].cpu().numpy()
    want = orc.correlator(L, F["u"][0], F["d"][0], F["s"][0], ch) * 2.0 ** (6 * e)
    assert np.isfinite(got).all()
    assert _err(got, want).max() < 2e-5
    cor.close()


def test_odd_T_and_ragged_slot_batches():
    """T = 5 slices through 2 slots per build: the last build holds one."""
    L, T = 4, 5
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, 3, 0.3, 0.4, seed=82)
    ch = [1, 16]
    cor = bbc.Correlators(L, T, 3, 0.3, 0.4, channels=ch, slices=2, device=dev)
    got = cor.run(torch.from_numpy(F["u"]).to(dev), torch.from_numpy(F["s"]).to(dev), range(T)).cpu().numpy()
    for t in range(T):
        want = orc.normalise(orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], ch), ch, (t - 3) % T, 0.3, 0.4)
        assert _err(got[t], want).max() < 1e-12, t
    cor.close()
