"""The C-ABI library loads, exports every entry point of include/bbc.h and
rejects bad arguments with the documented status codes (CPU only: no call
here touches a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1510_00903_gb300 import bbc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(bbc_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol():
    lib = ctypes.CDLL(bbc.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
        assert hasattr(bbc, n), n  # the binding keeps the C names


@pytest.mark.parametrize("L,T,t0,ch,prec", [
    (5, 8, 0, [0], 0), (16, 0, 0, [0], 0), (16, 8, 8, [0], 0),
    (16, 8, 0, [406], 0), (16, 8, 0, [-1], 0), (16, 8, 0, [3, 3], 0), (16, 8, 0, [0], 7)])
def test_create_rejects_bad_arguments(L, T, t0, ch, prec):
    with pytest.raises(bbc.BBCError) as e:
        bbc.bbc_create(L, T, t0, 0.3, 0.4, prec, ch)
    assert e.value.status == bbc.BBC_EINVAL
    assert bbc.bbc_last_error(None)


def test_workspace_and_state_errors():
    c = bbc.bbc_create(4, 4, 0, 0.3, 0.4, bbc.BBC_FP64, [0, 1])
    try:
        one, two = bbc.bbc_workspace_size(c, 1), bbc.bbc_workspace_size(c, 2)
        assert two > one > 0
        with pytest.raises(bbc.BBCError) as e:
            bbc.bbc_build_blocks(c, 1)
        assert e.value.status == bbc.BBC_ESTATE
        with pytest.raises(bbc.BBCError) as e:
            bbc.bbc_set_workspace(c, 256, one - 1, 1)
        assert e.value.status == bbc.BBC_ENOMEM
        with pytest.raises(bbc.BBCError) as e:
            bbc.bbc_set_workspace(c, 255, one, 1)
        assert e.value.status == bbc.BBC_EINVAL
    finally:
        bbc.bbc_destroy(c)


def test_mixed_workspace_is_smaller():
    a = bbc.bbc_create(16, 4, 0, 0.3, 0.4, bbc.BBC_FP64, list(range(52)))
    b = bbc.bbc_create(16, 4, 0, 0.3, 0.4, bbc.BBC_MIXED_FP32, list(range(52)))
    try:
        assert bbc.bbc_workspace_size(b, 1) < bbc.bbc_workspace_size(a, 1)
    finally:
        bbc.bbc_destroy(a)
        bbc.bbc_destroy(b)


def test_project_rejects_bad_arguments():
    """Argument checks of bbc_project run before any device work."""
    c = bbc.bbc_create(4, 4, 0, 0.3, 0.4, bbc.BBC_FP64, [0])
    try:
        n = 2 * 64 * 16 * 16  # bytes of two fields at L = 4
        for args in [(1 << 20, 2, None, None),             # no output
                     (1 << 20, 2, (1 << 20) + n - 16, None),  # R overlaps C
                     (1 << 20, 2, None, 1 << 20),           # Ra1 is C
                     (1 << 20, 2, 1 << 24, (1 << 24) + 256),  # R overlaps Ra1
                     ((1 << 20) + 8, 2, 1 << 24, None),     # misaligned
                     (1 << 20, -1, 1 << 24, None)]:         # negative count
            with pytest.raises(bbc.BBCError) as e:
                bbc.bbc_project(c, *args)
            assert e.value.status == bbc.BBC_EINVAL, args
    finally:
        bbc.bbc_destroy(c)


def test_tuning_defaults_validation_and_autotune_state():
    """Launch configurations: defaults, rejected shapes, and the autotuner's
    state checks (no device work here).  Mixed FP32 runs the tensor-core
    contraction (its CUDA-core kernel: 4 or 8 warps, two CTAs per SM); the
    bfloat16 trial runs the fused CUDA-core kernel (8, 12 or 16 warps)."""
    c = bbc.bbc_create(8, 4, 0, 0.3, 0.4, bbc.BBC_MIXED_FP32, [0, 1])
    b = bbc.bbc_create(8, 4, 0, 0.3, 0.4, bbc.BBC_MIXED_BF16, [0, 1])
    f = bbc.bbc_create(8, 4, 0, 0.3, 0.4, bbc.BBC_FP64, [0, 1])
    try:
        assert bbc.bbc_get_tuning(c) == {"build_sites": 1, "build_threads": 256, "fused_warps": 8, "fused_chunk": 18,
                                         "fused_steps": 1, "pair_groups": 48, "tc_kernel": 0}
        bbc.bbc_set_tuning(c, 2, 256, 4, 36, 2)  # no workspace yet: host schedule only
        assert bbc.bbc_get_tuning(c) == {"build_sites": 2, "build_threads": 256, "fused_warps": 4, "fused_chunk": 36,
                                         "fused_steps": 2, "pair_groups": 48, "tc_kernel": 0}
        # the trace-form products on mma.sync (1) or tcgen05 (0); nothing else
        bbc.bbc_set_tuning(c, 2, 256, 4, 36, 2, tc_kernel=1)
        assert bbc.bbc_get_tuning(c)["tc_kernel"] == 1
        with pytest.raises(bbc.BBCError) as e:
            bbc.bbc_set_tuning(c, 2, 256, 4, 36, 2, tc_kernel=2)
        assert e.value.status == bbc.BBC_EINVAL
        bbc.bbc_set_tuning(c, 2, 256, 4, 36, 2, tc_kernel=0)
        # the dense-tuple FP32 build runs one or two sites per CTA of 256 or 512 threads
        for bad in [(3, 256, 8, 18), (4, 256, 8, 18), (4, 512, 8, 18),
                    (1, 256, 10, 18), (1, 256, 8, 20), (1, 256, 8, 18, 2), (1, 256, 4, 18, 3), (1, 256, 16, 18),
                    (1, 256, 12, 18)]:
            with pytest.raises(bbc.BBCError) as e:
                bbc.bbc_set_tuning(c, *bad)
            assert e.value.status == bbc.BBC_EINVAL, bad
        assert bbc.bbc_get_tuning(c)["fused_chunk"] == 36  # a rejected set leaves the configuration
        assert bbc.bbc_get_tuning(b) == {"build_sites": 1, "build_threads": 256, "fused_warps": 16, "fused_chunk": 18,
                                         "fused_steps": 1, "pair_groups": 48, "tc_kernel": 0}
        bbc.bbc_set_tuning(b, 1, 256, 16, 18, 1, tc_kernel=1)  # no tensor-core kernel here: ignored
        assert bbc.bbc_get_tuning(b)["tc_kernel"] == 0
        bbc.bbc_set_tuning(b, 2, 256, 12, 36, 2)
        for bad in [(1, 256, 16, 18, 2), (1, 256, 8, 18, 3), (1, 256, 4, 18)]:
            with pytest.raises(bbc.BBCError) as e:
                bbc.bbc_set_tuning(b, *bad)
            assert e.value.status == bbc.BBC_EINVAL, bad
        # FP64 blocks of four sites need 365 KB of shared memory: not valid
        with pytest.raises(bbc.BBCError):
            bbc.bbc_set_tuning(f, 4, 512)
        bbc.bbc_set_tuning(f, 2, 256, 8, 7)  # fused fields ignored for FP64
        assert bbc.bbc_get_tuning(f)["fused_warps"] == 16
        with pytest.raises(bbc.BBCError) as e:
            bbc.bbc_autotune(c)
        assert e.value.status == bbc.BBC_ESTATE
    finally:
        bbc.bbc_destroy(c)
        bbc.bbc_destroy(b)
        bbc.bbc_destroy(f)


def test_launch_counts_follow_the_path():
    """Kernel launches per call: the tensor-core path runs two contraction
    kernels, the fused CUDA-core path one, the FP64 path two (products and
    Wick sums); the q-major layout fuses the x and y FFT passes up to L = 32
    and runs the forward transform there as one queue-driven launch."""
    want = {bbc.BBC_MIXED_FP32: (2, 2, 5), bbc.BBC_MIXED_TF32: (2, 2, 5), bbc.BBC_MIXED_BF16: (2, 3, 4),
            bbc.BBC_FP64: (2, 4, 6), bbc.BBC_DF64: (2, 4, 6)}
    for prec, (load, build, contract) in want.items():
        c = bbc.bbc_create(16, 4, 0, 0.3, 0.4, prec, list(range(52)))
        try:
            assert bbc.bbc_launch_counts(c) == {"load": load, "build": build, "contract": contract}, prec
        finally:
            bbc.bbc_destroy(c)
    # L = 48: three forward passes of the q-major layout, no queue-driven launch
    c = bbc.bbc_create(48, 4, 0, 0.3, 0.4, bbc.BBC_MIXED_FP32, list(range(52)))
    try:
        assert bbc.bbc_launch_counts(c) == {"load": 2, "build": 4, "contract": 6}
    finally:
        bbc.bbc_destroy(c)


def test_bounded_wait_entry_points_without_a_workspace():
    """bbc_device_status is OK before anything ran; the bounded-wait self-test
    checks its limit (EINVAL) and needs a workspace (ESTATE), with no CUDA call."""
    c = bbc.bbc_create(8, 4, 0, 0.3, 0.4, bbc.BBC_MIXED_FP32, list(range(52)))
    try:
        bbc.bbc_device_status(c)
        assert bbc.bbc_check_bounded_wait(c, 0) == bbc.BBC_EINVAL
        assert bbc.bbc_check_bounded_wait(c, (1 << 22) + 1) == bbc.BBC_EINVAL
        assert bbc.bbc_check_bounded_wait(c, 1000) == bbc.BBC_ESTATE
        assert "workspace" in bbc.lib().bbc_last_error(c).decode()
    finally:
        bbc.bbc_destroy(c)


def test_lower_components_plan_and_errors():
    """The lower spin components give a plan of the same shape (the C gamma5
    block swap maps one onto the other); a bad component selector is EINVAL."""
    ch = list(range(52))
    up = bbc.bbc_create(16, 32, 0, 0.3, 0.4, bbc.BBC_FP64, ch)
    lo = bbc.bbc_create_components(16, 32, 0, 0.3, 0.4, bbc.BBC_FP64, ch, bbc.BBC_LOWER)
    try:
        assert bbc.bbc_plan_sizes(lo) == bbc.bbc_plan_sizes(up)
        assert bbc.bbc_plan_sizes(lo)["block_outputs"] == 7368
        assert bbc.bbc_workspace_size(lo, 1) == bbc.bbc_workspace_size(up, 1)
    finally:
        bbc.bbc_destroy(up)
        bbc.bbc_destroy(lo)
    with pytest.raises(bbc.BBCError) as e:
        bbc.bbc_create_components(4, 4, 0, 0.3, 0.4, bbc.BBC_FP64, [0], 2)
    assert e.value.status == bbc.BBC_EINVAL


def test_batch_and_check_argument_errors():
    """bbc_batch_run rejects an empty batch and names a bad item; unknown
    check flags are EINVAL (no device work)."""
    items = (bbc.bbc_batch_item * 2)()
    with pytest.raises(bbc.BBCError) as e:
        bbc.bbc_batch_run(items, 0)
    assert e.value.status == bbc.BBC_EINVAL
    with pytest.raises(bbc.BBCError) as e:
        bbc.bbc_batch_run(items, 2)  # item 0 has no context
    assert e.value.status == bbc.BBC_EINVAL and "item 0" in str(e.value)
    c = bbc.bbc_create(4, 4, 0, 0.3, 0.4, bbc.BBC_FP64, [0])
    try:
        bbc.bbc_set_checks(c, bbc.BBC_CHECK_INPUT | bbc.BBC_CHECK_OUTPUT)
        with pytest.raises(bbc.BBCError) as e:
            bbc.bbc_set_checks(c, 4)
        assert e.value.status == bbc.BBC_EINVAL
    finally:
        bbc.bbc_destroy(c)


def test_bf16_trial_rejects_channel_lists_beyond_the_fused_kernel():
    """The bfloat16 trial runs only in the fused contraction; all 52 octet
    channels with the 90 decuplet ids need more shared memory than one CTA
    has (the FP32 path then takes the unfused route, which is accepted).
    The 90 decuplet ids alone fit."""
    big = bbc.CHANNELS_52 + bbc.OMEGA_OMEGA + bbc.P_OMEGA
    with pytest.raises(bbc.BBCError) as e:
        bbc.bbc_create(4, 4, 0, 0.3, 0.4, bbc.BBC_MIXED_BF16, big)
    assert e.value.status == bbc.BBC_EINVAL and "BBC_MIXED_FP32" in str(e.value)
    for prec, chans in ((bbc.BBC_MIXED_FP32, big), (bbc.BBC_MIXED_BF16, bbc.OMEGA_OMEGA + bbc.P_OMEGA)):
        c = bbc.bbc_create(4, 4, 0, 0.3, 0.4, prec, chans)
        bbc.bbc_destroy(c)


def test_tuning_pair_groups():
    """pair_groups defaults to 48 (192 for double-float) and takes 48, 96, 192
    or 384; other values are rejected (CPU: no workspace attached)."""
    c = bbc.bbc_create(4, 4, 0, 0.3, 0.4, bbc.BBC_FP64, [0, 1])
    d = bbc.bbc_create(4, 4, 0, 0.3, 0.4, bbc.BBC_DF64, [0, 1])
    try:
        assert bbc.bbc_get_tuning(c)["pair_groups"] == 48
        assert bbc.bbc_get_tuning(d)["pair_groups"] == 192
        bbc.bbc_set_tuning(c, 1, 256, pair_groups=96)
        assert bbc.bbc_get_tuning(c)["pair_groups"] == 96
        with pytest.raises(bbc.BBCError) as e:
            bbc.bbc_set_tuning(c, 1, 256, pair_groups=64)
        assert e.value.status == bbc.BBC_EINVAL
        assert bbc.bbc_get_tuning(c)["pair_groups"] == 96
    finally:
        bbc.bbc_destroy(c)
        bbc.bbc_destroy(d)


def test_tuning_cache_file(tmp_path):
    """The autotune cache: keyed by GPU model and problem, JSON round trip,
    atomic replace, a missing or broken file reads as empty, and a cached
    configuration applies to a context (CPU: no workspace needed)."""
    path = str(tmp_path / "tune.json")
    assert bbc.tuning_cache_load(path) == {}
    k1 = bbc.tuning_cache_key("GB300", 16, bbc.BBC_FP64, bbc.BBC_UPPER, range(52))
    k2 = bbc.tuning_cache_key("GB300", 16, bbc.BBC_MIXED_FP32, bbc.BBC_UPPER, range(52))
    assert k1 != k2 and k1 != bbc.tuning_cache_key("B200", 16, bbc.BBC_FP64, bbc.BBC_UPPER, range(52))
    cfg = {"build_sites": 2, "build_threads": 256, "fused_warps": 16, "fused_chunk": 18, "fused_steps": 1,
           "pair_groups": 96}
    bbc.tuning_cache_store(path, k1, cfg)
    bbc.tuning_cache_store(path, k2, dict(cfg, fused_chunk=72))
    data = bbc.tuning_cache_load(path)
    assert data[k1] == cfg and data[k2]["fused_chunk"] == 72
    assert not any(n.startswith("tune.json.tmp") for n in os.listdir(tmp_path))
    c = bbc.bbc_create(4, 4, 0, 0.3, 0.4, bbc.BBC_FP64, [0, 1])
    try:
        bbc.bbc_set_tuning(c, **{k: v for k, v in data[k1].items()})
        assert bbc.bbc_get_tuning(c)["pair_groups"] == 96 and bbc.bbc_get_tuning(c)["build_sites"] == 2
    finally:
        bbc.bbc_destroy(c)
    with open(path, "w") as f:
        f.write("{not json")
    assert bbc.tuning_cache_load(path) == {}


def test_plan_export_arguments():
    """bbc_plan_export: EINVAL without a context or sizes array; sizes alone
    when any table pointer is NULL (nothing else is written)."""
    import numpy as np
    assert bbc.lib().bbc_plan_export(None, None, None, None, None, None, None, None) == bbc.BBC_EINVAL
    c = bbc.bbc_create(4, 4, 0, 0.3, 0.4, bbc.BBC_FP64, [0, 1])
    try:
        assert bbc.lib().bbc_plan_export(c, None, None, None, None, None, None, None) == bbc.BBC_EINVAL
        sizes = np.zeros(5, dtype=np.int32)
        row_ptr = np.full(8, -7, dtype=np.int32)
        assert bbc.lib().bbc_plan_export(c, sizes.ctypes.data, row_ptr.ctypes.data, None, None, None, None,
                                         None) == bbc.BBC_OK
        assert sizes[0] == bbc.bbc_plan_sizes(c)["block_outputs"] and np.all(row_ptr == -7)
        # capacities too small: nothing is written, EINVAL, the needed sizes come back
        need = sizes.copy()
        small = need.copy()
        small[1] -= 1
        arrays = [np.full(int(need[0]) + 1, -7, np.int32), np.zeros((int(need[1]), 3), np.int32),
                  np.zeros((int(need[2]), 24), np.int32), np.zeros(int(need[4]) + 1, np.int32),
                  np.zeros(int(need[3]), np.int32), np.zeros(int(need[3]), np.float64)]
        assert bbc.lib().bbc_plan_export(c, small.ctypes.data, *(a.ctypes.data for a in arrays)) == bbc.BBC_EINVAL
        assert np.array_equal(small, need) and np.all(arrays[0] == -7)
        p = bbc.bbc_plan_export(c)
        assert p["row_ptr"][0] == 0 and p["row_ptr"][-1] == len(p["terms"]) == sizes[1]
        assert p["out_ptr"][-1] == len(p["items"]) == sizes[3] and len(p["out_ptr"]) == 2 * 16 + 1
    finally:
        bbc.bbc_destroy(c)


def test_static_entry_point_argument_checks():
    """bbc_run_slice_static rejects, before any device work: other precisions,
    contexts with numeric checks, and misaligned pointers."""
    fake = 1 << 20  # 16-byte aligned stand-ins: never dereferenced on these paths
    t = bbc.bbc_create(4, 4, 0, 0.3, 0.4, bbc.BBC_MIXED_TF32, [0])
    c = bbc.bbc_create(4, 4, 0, 0.3, 0.4, bbc.BBC_FP64, [0])
    try:
        with pytest.raises(bbc.BBCError) as e:
            bbc.bbc_run_slice_static(t, 1, fake, fake, bbc.BBC_C128, fake, True)
        assert e.value.status == bbc.BBC_EINVAL and "BBC_FP64" in str(e.value)
        bbc.bbc_set_checks(c, bbc.BBC_CHECK_OUTPUT)
        with pytest.raises(bbc.BBCError) as e:
            bbc.bbc_run_slice_static(c, 1, fake, fake, bbc.BBC_C128, fake, True)
        assert e.value.status == bbc.BBC_EINVAL and "numeric checks" in str(e.value)
        bbc.bbc_set_checks(c, 0)
        with pytest.raises(bbc.BBCError) as e:
            bbc.bbc_run_slice_static(c, 1, fake + 8, fake, bbc.BBC_C128, fake, True)
        assert e.value.status == bbc.BBC_EINVAL
    finally:
        bbc.bbc_destroy(t)
        bbc.bbc_destroy(c)
