"""The no-allocation entry point bbc_run_slice_static against the regular
path (workspace-backed bbc_load_propagator / bbc_build_blocks / bbc_contract).

bbc_run_slice_static serves callers that cannot allocate device memory
(their process's device memory belongs to another runtime's pool allocator,
or the call sits on a loop that must not take an allocation); all its
scratch lives in a static array inside libbbc.  This file is collected last
so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1510_00903_gb300 import bbc  # noqa: E402

TOL = {bbc.BBC_FP64: 1e-12, bbc.BBC_MIXED_FP32: 2e-5}


@pytest.mark.parametrize("precision", [bbc.BBC_FP64, bbc.BBC_MIXED_FP32])
def test_static_scratch_matches_workspace_path_twice(precision):
    L, T, t0 = 4, 6, 1
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, t0, 0.3, 0.4, seed=21)
    chans = list(range(52))
    times = [2, 5]
    Sl = torch.from_numpy(F["u"][times]).to(dev)
    Ss = torch.from_numpy(F["s"][times]).to(dev)
    ref = bbc.Correlators(L, T, t0, 0.3, 0.4, channels=chans, precision=precision, device=dev)
    want = ref.run(Sl, Ss, times, normalised=True)
    torch.cuda.synchronize(dev)
    ref.close()
    # a context without any workspace: planning only
    stream = torch.cuda.current_stream(dev)
    ctx = bbc.bbc_create(L, T, t0, 0.3, 0.4, precision, chans, stream.cuda_stream)
    try:
        for i, t in enumerate(times):  # two calls in a row on the shared array
            out = torch.full((len(chans), L ** 3, 16), float("nan"), dtype=torch.complex128, device=dev)
            bbc.bbc_run_slice_static(ctx, t, Sl[i].data_ptr(), Ss[i].data_ptr(), bbc.BBC_C128, out.data_ptr(), True)
            torch.cuda.synchronize(dev)
            got = out.cpu().numpy()
            w = want[i].cpu().numpy()
            scale = np.abs(w).reshape(len(chans), -1).max(axis=1)
            err = np.abs(got - w).reshape(len(chans), -1).max(axis=1) / np.where(scale > 0, scale, 1.0)
            assert np.isfinite(got).all()
            assert err.max() < TOL[precision], (t, err.max())
    finally:
        bbc.bbc_destroy(ctx)


def test_static_scratch_rejects_large_lattice():
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = bbc.bbc_create(8, 2, 0, 0.3, 0.4, bbc.BBC_FP64, list(range(52)), torch.cuda.current_stream(dev).cuda_stream)
    try:
        S = torch.zeros((8 ** 3, 12, 12), dtype=torch.complex128, device=dev)
        out = torch.zeros((52, 8 ** 3, 16), dtype=torch.complex128, device=dev)
        with pytest.raises(bbc.BBCError) as e:
            bbc.bbc_run_slice_static(ctx, 0, S.data_ptr(), S.data_ptr(), bbc.BBC_C128, out.data_ptr(), True)
        assert e.value.status == bbc.BBC_EINVAL
        assert "static" in str(e.value)
    finally:
        bbc.bbc_destroy(ctx)
