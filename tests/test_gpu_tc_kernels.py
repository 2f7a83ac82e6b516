"""The two tensor-core kernels of the mixed contraction (GPU), both against the
FP64 path (pinned to the oracle elsewhere): the trace-form products on tcgen05
(tuning tc_kernel 0: one persistent CTA per SM, TMEM accumulators) and on
mma.sync (tc_kernel 1, whose CUDA-core kernel runs beside it on a second
stream from 4096 pairs {q, -q} on).  L = 8 is one wave of pairs; L = 24
(13824 sites) takes the two-stream pipeline in four chunks and gives the
persistent kernel many pairs per CTA.  The channel lists give G of 12, 24,
48 and 52 blocks (padded to 16, 32, 48 and 64: every warp-task count of the
tcgen05 kernel, and N = 128 with no unstaged rows of A).  Both kernels compute
the same G up to the order of FP32 accumulation.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1510_00903_gb300 import bbc  # noqa: E402

MIXED_TOL = 2e-5


def _err(got, want):
    scale = np.abs(want).max(axis=(-2, -1), keepdims=True)
    return (np.abs(got - want) / scale).max()


@pytest.mark.parametrize("L,chans", [(8, list(range(52))), (24, [0, 10, 27, 51]), (8, [0]), (8, [1]),
                                     (8, list(range(52)) + [154])])
def test_both_tensor_core_kernels_match_fp64(L, chans):
    dev = torch.device("cuda", torch.cuda.current_device())
    T, t = 4, 2
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=131 + L, times=[t])
    Sl = torch.from_numpy(F["u"]).to(dev)
    Ss = torch.from_numpy(F["s"]).to(dev)
    ref = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=chans, precision=bbc.BBC_FP64, device=dev)
    want = ref.run(Sl, Ss, [t]).cpu().numpy()
    ref.close()
    got = {}
    for kernel in (0, 1):
        cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=chans, precision=bbc.BBC_MIXED_FP32, device=dev)
        cfg = cor.tuning()
        cor.set_tuning(dict(cfg, tc_kernel=kernel))
        assert cor.tuning()["tc_kernel"] == kernel
        got[kernel] = cor.run(Sl, Ss, [t]).cpu().numpy()
        cor.status()
        cor.close()
        assert _err(got[kernel], want) < MIXED_TOL, kernel
    assert _err(got[0], got[1]) < 1e-5
