"""Host-side helpers of the benchmark (CPU only): the DRAM-traffic lookup in
an ncu summary and the thread count the oracle timing reports."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle.oracle as orc  # noqa: E402


def _summary(tmp_path, sha, items, dram="123456"):
    p = tmp_path / "summary.md"
    p.write_text("# k\n\n| metric | value |\n|---|---|\n\n"
                 f"- kernels_cu_sha256: {sha}\n- pair_items_per_q: {items}\n- dram_bytes_per_launch: {dram}\n")
    return str(p)


def test_profiled_traffic_needs_the_same_kernel_and_plan(tmp_path):
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    assert bench.profiled_traffic(_summary(tmp_path, sha, 2448), str(src), 2448) == 123456.0
    # another plan size, another kernel source, no summary: no traffic figure
    assert bench.profiled_traffic(_summary(tmp_path, sha, 4080), str(src), 2448) is None
    assert bench.profiled_traffic(_summary(tmp_path, "0" * 64, 2448), str(src), 2448) is None
    assert bench.profiled_traffic(str(tmp_path / "missing.md"), str(src), 2448) is None


def test_committed_pair_products_summary_has_the_fields():
    text = open(os.path.join(ROOT, "profiles", "k_pair_products_f64_L16_slice.md")).read()
    for key in ("kernels_cu_sha256:", "pair_items_per_q:", "dram_bytes_per_launch:"):
        assert key in text, key


def test_roofline_denominators():
    # FP64 pipe: 152 SMs x 2 FMA x 2 flop x 2070 MHz; complex MAC = 3 FMAs for 8 flops
    assert abs(bench.FP64_PEAK_TFLOPS - 1.2586) < 1e-3
    assert abs(bench.FP64_CMAC_PEAK_TFLOPS - 1.6781) < 1e-3
    assert abs(bench.FP32_PEAK_TFLOPS - 80.54) < 1e-2


def test_oracle_reports_its_threads():
    n = orc.threads()
    assert 1 <= n <= (os.cpu_count() or 1) * 4


def test_hbm_peak_from_the_peaks_file(tmp_path):
    f = tmp_path / "peaks.json"
    f.write_text('{"hbm_gbs": 7000.5, "bf16_tflops": 1945.0}')
    assert bench.measured_hbm_gbs(str(f))[0] == 7000.5
    f.write_text("{}")
    assert bench.measured_hbm_gbs(str(f))[0] == 6803.8
    assert bench.measured_hbm_gbs(str(tmp_path / "none.json"))[0] == 6803.8


def test_step_roofline_of_the_52_channel_plan():
    """Work counts of the bench plan and the stage-wise floor of an FP64 step."""
    from paper_1510_00903_gb300 import bbc
    ctx = bbc.bbc_create(16, 32, 0, 0.3, 0.4, bbc.BBC_FP64, list(range(52)))
    try:
        counts = bench.plan_counts(bbc.bbc_plan_export(ctx), bbc.bbc_plan_sizes(ctx))
    finally:
        bbc.bbc_destroy(ctx)
    assert counts["block_rows"] == 7368 and counts["row_terms"] == 33816 and counts["outputs"] == 52 * 16
    assert counts["diquarks"] == 2  # (l l) and (l s) C gamma5: octet families only
    assert 0 < counts["tensor_entries"] <= 2 * 1728 * 4
    assert counts["pair_items"] == 16 * (counts["pair_items"] // 16) and counts["wick_terms"] > 0
    V, T = 16 ** 3, 32
    stage_ms = {"ingest": 2.0, "build": 60.0, "fft_fwd": 50.0, "contract": 120.0, "wick": 3.0, "fft_inv": 7.0,
                "normalise": 0.1, "project": 0.0}
    r = bench.step_roofline(counts, V, T, stage_ms, 250.0, hbm_gbs=6800.0)
    st = r["stages"]
    # the contraction: three FP64 FMAs per complex multiply-add on 152 SMs x 2 FMA/clk x 2.07 GHz
    want = 3.0 * counts["pair_macs"] * V * T / (152 * 2 * 2.070e9) * 1e3
    assert abs(st["contract"]["floor_ms"] - want) < 1e-9 * want and st["contract"]["bound"] == "fp64"
    # ingest moves 2 x 144 complex128 values in and out per site: copy-bandwidth bound
    want = 2 * 144 * 32 * V * T / 6800e9 * 1e3
    assert abs(st["ingest"]["floor_ms"] - want) < 1e-9 * want and st["ingest"]["bound"] == "hbm"
    assert abs(r["floor_ms"] - sum(s["floor_ms"] for s in st.values())) < 1e-9
    assert abs(r["frac"] - r["floor_ms"] / 250.0) < 1e-12
    assert all(abs(s["frac"] - s["floor_ms"] / stage_ms[k]) < 1e-12 for k, s in st.items())


def test_step_roofline_mixed_routes():
    """Mixed precision: the fused contraction (no Wick stage timed) is one
    stage bounded by the FP32 products, the FP64 sums or the traffic; the
    unfused route has products and sums as two stages."""
    counts = {"block_rows": 7368, "row_terms": 33816, "tensor_entries": 8880, "diquarks": 2, "pair_macs": 174208,
              "pair_items": 2448, "wick_terms": 5504, "outputs": 832}
    V, T = 16 ** 3, 32
    fused = {"ingest": 2.0, "build": 11.0, "fft_fwd": 6.0, "contract": 15.0, "fft_inv": 2.7, "wick": 0.0}
    r = bench.step_roofline(counts, V, T, fused, 40.0, mixed=True, hbm_gbs=6800.0)
    st = r["stages"]
    assert "wick" not in st
    fp32 = 8.0 * 174208 * V * T / (bench.FP32_PEAK_TFLOPS * 1e12) * 1e3
    fp64 = 4.0 * 5504 * V * T / (bench.FP64_PEAK_TFLOPS * 1e12) * 1e3
    hbm = (7368 * 8 + 832 * 16) * V * T / 6800e9 * 1e3
    assert abs(st["contract"]["floor_ms"] - max(fp32, fp64, hbm)) < 1e-12
    assert st["fft_fwd"]["bound"] == "hbm"  # FP32 transforms of 8-byte values
    unfused = dict(fused, wick=3.0)
    st = bench.step_roofline(counts, V, T, unfused, 45.0, mixed=True, hbm_gbs=6800.0)["stages"]
    assert abs(st["wick"]["floor_ms"] - max(fp64, (2448 * 8 + 832 * 16) * V * T / 6800e9 * 1e3)) < 1e-12
    assert st["contract"]["bound"] in ("fp32", "hbm")
