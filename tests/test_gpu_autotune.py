"""Autotuner and every launch configuration of the block build and the fused
contraction: each gives the oracle's correlators (GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
import oracle.oracle as orc

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1510_00903_gb300 import bbc  # noqa: E402

BUILD = [(1, 256), (2, 256), (2, 512), (4, 512), (1, 512)]
MIXED_TOL = 2e-5


def _err(got, want):
    scale = np.abs(want).reshape(want.shape[0], -1).max(axis=1)
    return (np.abs(got - want).reshape(want.shape[0], -1).max(axis=1) / scale).max()


@pytest.mark.parametrize("precision", [bbc.BBC_FP64, bbc.BBC_MIXED_FP32])
def test_autotune_then_oracle(precision):
    L, T, t = 8, 4, 1
    chans = [0, 10, 51]
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=77)
    Sl, Ss = torch.from_numpy(F["u"]).to(dev), torch.from_numpy(F["s"]).to(dev)
    cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=chans, precision=precision, device=dev)
    cfg, ms = cor.autotune(Sl[0], Ss[0], t=0, reps=2)
    # FP64: four pair_groups candidates; mixed (tensor cores): the CUDA-core
    # kernel's (warps, steps) shapes x 5 chunks, then the tcgen05 and the
    # mma.sync tensor-core kernels
    n_second = 4 if precision == bbc.BBC_FP64 else 15 + 2
    assert len(ms) == len(BUILD) + n_second
    assert all(v > 0 for v in ms[len(BUILD):])
    assert cfg["pair_groups"] in (48, 96, 192, 384)
    assert cfg["tc_kernel"] in (0, 1)
    assert (cfg["build_sites"], cfg["build_threads"]) in BUILD
    if precision != bbc.BBC_FP64:  # the dense-tuple FP32 build runs 1 or 2 sites per CTA of 256 or 512 threads
        assert all((v == -1) == (BUILD[i][0] == 4) for i, v in enumerate(ms[:len(BUILD)]))
    # a later context for the same problem starts with the tuned configuration
    cor2 = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=chans, precision=precision, device=dev)
    assert cor2.tuning() == cfg
    cor2.close()
    out = cor.run(Sl[t:t + 1], Ss[t:t + 1], [t])[0].cpu().numpy()
    want = orc.normalise(orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], chans), chans, t, 0.3, 0.4)
    assert _err(out, want) < (1e-12 if precision == bbc.BBC_FP64 else MIXED_TOL)
    cor.close()


@pytest.mark.parametrize("precision", [bbc.BBC_FP64, bbc.BBC_MIXED_FP32, bbc.BBC_MIXED_BF16])
def test_every_configuration_matches(precision):
    L, T, t = 8, 4, 2
    chans = [1, 14, 41]
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=78)
    Sl, Ss = torch.from_numpy(F["u"][t:t + 1]).to(dev), torch.from_numpy(F["s"][t:t + 1]).to(dev)
    want = orc.normalise(orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], chans), chans, t, 0.3, 0.4)
    cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=chans, precision=precision, device=dev)
    ref = None
    # mixed FP32: the tensor-core path's CUDA-core kernel; bfloat16: the fused kernel
    shapes = [(4, 1), (4, 2), (8, 1)] if precision == bbc.BBC_MIXED_FP32 else [(8, 1), (8, 2), (12, 1), (12, 2), (16, 1)]
    tol = {bbc.BBC_FP64: 1e-12, bbc.BBC_MIXED_FP32: MIXED_TOL, bbc.BBC_MIXED_BF16: 2e-2}[precision]
    # FP64: every pair_groups value (the fused fields are ignored there)
    fused = [(16, 18, 1, g) for g in (48, 96, 192, 384)] if precision == bbc.BBC_FP64 else \
        [(w, k, st, 48) for w, st in shapes for k in (0, 18, 36, 72, 144)]
    tried = 0
    for sites, threads in BUILD:
        for warps, chunk, steps, groups in fused:
            try:
                cor.set_tuning({"build_sites": sites, "build_threads": threads, "fused_warps": warps,
                                "fused_chunk": chunk, "fused_steps": steps, "pair_groups": groups})
            except bbc.BBCError:
                # FP64: four sites need 365 KB of shared memory; FP32 (dense-tuple
                # build): one or two sites per CTA
                assert sites == 4
                continue
            out = cor.run(Sl, Ss, [t])[0].cpu().numpy()
            assert _err(out, want) < tol, (sites, threads, warps, chunk, steps, groups)
            if precision == bbc.BBC_FP64:
                # the build sums every row in the same order whatever the shape, and
                # a task's products do not depend on the list it is in
                if ref is None:
                    ref = out
                assert np.array_equal(out, ref)
            tried += 1
    assert tried == {bbc.BBC_FP64: 16, bbc.BBC_MIXED_FP32: 60, bbc.BBC_MIXED_BF16: 100}[precision]
    cor.close()
