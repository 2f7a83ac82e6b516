#!/usr/bin/env python
"""Benchmark of the effective block algorithm on GB300.

Workload (one step): all 52 octet baryon-baryon channels of Sec. 4 on an
L^3 x T = 16^3 x 32 lattice with one wall source at t0 = 0 -- every time slice
through propagator ingest, block build, forward FFT, q-space contraction,
inverse FFT and normalisation.  Synthetic complex128 propagators (i.i.d.
unit complex Gaussians x exp(-m_f |t - t0|), m_ud = 0.3, m_s = 0.4), resident
in HBM before the timed region.  Headline: plain FP64 path; the mixed path
(FP32 blocks/FFTs/pair products, FP64 Wick-sign sums) is reported beside it.

Metric: site*channels/s = (#ranks) x L^3 x T x 52 / seconds per step.
Multi-GPU (torchrun): every rank runs the same workload on its own wall
source (independent units, weak scaling, no collective on the data path).

``--impl reference`` times the CPU FP64 oracle (the reference of this
build) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

L_BENCH, T_BENCH, N_CH = 16, 32, 52
M_UD, M_S = 0.3, 0.4
#: paper's best elapsed time for this workload: 16^3 x 32, 52 channels, 19 s
#: on 32 BlueGene/Q nodes (Sec. 5, Table ElapsedTime, 4x8 and 2x16 splits)
PAPER_SITE_CH_PER_S = 16 ** 3 * 32 * 52 / 19.0
#: FP64 FMA peak derived from unit counts and clocks: 152 SMs x 2 FP64 FMA
#: per SM per clock x 2 flop x 2070 MHz (a probe measured 1.197 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
#: the same pipe's ceiling for complex multiply-adds, in the algorithmic
#: 8 flops each: a complex product takes at least three real multiplications
#: (Gauss), so at most 629 G FMA/s / 3 = 209.8 G complex MACs/s = 1.678 TFLOP/s
FP64_CMAC_PEAK_TFLOPS = FP64_PEAK_TFLOPS * 8.0 / 6.0
CMAC_PEAK_SOURCE = ("derived: 152 SM x 2 FP64 FMA/clk x 2070 MHz = 629.3 G FMA/s; a complex multiply-add (8 "
                    "algorithmic flops) needs at least 3 real FMAs (three-multiplication complex product), so the "
                    "FP64 pipe's ceiling is 209.8 G complex MACs/s = 1.678 TFLOP/s")
#: FP32 FMA peak: 152 SMs x 128 lanes x 2 flop x 2070 MHz (probe: 74.8 TFLOP/s)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def measured_hbm_gbs(path=os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")):
    """STREAM-style copy bandwidth (GB/s) measured on this GPU model, from
    the peaks file beside this script; 6803.8 (the same measurement, taken
    earlier on a GB300) when the file is absent or has no such figure."""
    try:
        v = float(json.load(open(path))["hbm_gbs"])
        if v > 0:
            return v, "measured copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return 6803.8, "measured copy bandwidth of an earlier GB300 run (no MEASURED_PEAKS.json)"


HBM_PEAK_GBS, HBM_PEAK_SOURCE = measured_hbm_gbs()


def profiled_traffic(path, kernel_src, pair_items):
    """DRAM bytes per launch of the dominant kernel from a committed ncu
    summary, if the summary was taken on the current kernel source (its
    SHA-256 is recorded beside the counters) and on a plan of the same size
    (its block-pair products per q); else None."""
    import hashlib
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
    except OSError:
        return None
    fields = {}
    for line in text.splitlines():
        line = line.strip().lstrip("-* ").strip()
        if ":" in line and line.startswith(("kernels_cu_sha256", "dram_bytes_per_launch", "pair_items_per_q")):
            k, v = line.split(":", 1)
            fields[k.strip().strip("`")] = v.strip().strip("`")
    if fields.get("kernels_cu_sha256") != sha or "dram_bytes_per_launch" not in fields:
        return None
    if fields.get("pair_items_per_q") != str(pair_items):
        return None
    return float(fields["dram_bytes_per_launch"])


#: diquark kind read by each sink-tensor family (the families' Gamma1 and the
#: flavours of their first two quarks), in the plan's family order: the four
#: C gamma5 families on (l l) and (l s), (s s s) with C gamma_1, C gamma_2,
#: C gamma_3, then per flavour pattern (l l l), (l l s), (l s l), (l s s),
#: (s s l) the three vector diquarks (l l), (l s) or (s s)
_SS, _LL, _LS = (2, 3, 4), (5, 6, 7), (8, 9, 10)
FAMILY_DIQUARK = [0, 0, 1, 1, *_SS, *_LL, *_LL, *_LS, *_LS, *_SS]


def plan_counts(plan, sizes):
    """Algorithmic work counts of a plan, from its exported tables: block rows,
    their weighted terms, the distinct sink-tensor entries they read, the
    diquark kinds behind those, the block-pair complex multiply-adds and
    products per q, the signed Wick terms and the outputs (channel x spin)."""
    terms = plan["terms"]
    fams = {int(f) for f in terms[:, 0]}
    return {"block_rows": len(plan["row_ptr"]) - 1, "row_terms": int(len(terms)),
            "tensor_entries": len({(int(f), int(e)) for f, e in terms[:, :2]}),
            "diquarks": len({FAMILY_DIQUARK[f] for f in fams}),
            "pair_macs": int(sizes["pair_macs_per_site"]), "pair_items": int(sizes["pair_items"]),
            "wick_terms": int(len(plan["items"])), "outputs": len(plan["out_ptr"]) - 1}


def step_roofline(counts, V, slices, stage_ms, step_ms, mixed=False, hbm_gbs=None, fp64_tflops=FP64_PEAK_TFLOPS,
                  cmac_tflops=FP64_CMAC_PEAK_TFLOPS, fp32_tflops=FP32_PEAK_TFLOPS):
    """Stage-wise roofline of one step of `slices` time slices: per stage the
    larger of its algorithmic bytes over the copy bandwidth and its
    algorithmic flops over the pipe that runs them; the step's floor is the
    sum over stages and frac = floor / measured step time.

    Algorithmic work per slice (V sites), blocks as b-byte complex values
    (16 plain FP64, 8 mixed FP32), correlators and Wick sums 16-byte:
      ingest   2 x 144 complex128 values read, written as blocks' type;
      build    the propagators read, the block rows written; 432 entries x 8
               complex products per diquark kind, 3 complex multiply-adds per
               sink-tensor entry (8 flops each), 4 flops per weighted term;
      fft_fwd  one read and one write of every block field, 5 V log2 V flops each;
      contract the block fields read, the pair products written, 8 flops per
               complex multiply-add (FP64: over the pipe's complex-MAC ceiling);
      wick     the products read, the outputs written, 4 FP64 flops per signed term;
      fft_inv  the outputs read and the correlators written, 5 V log2 V flops each.
    Mixed precision with the fused contraction (no separate Wick stage
    timed): the contraction reads the block fields once and writes the
    outputs, its FP32 products and FP64 Wick sums bounded by their own pipes."""
    import math
    hbm = HBM_PEAK_GBS if hbm_gbs is None else hbm_gbs
    c, lg = counts, math.log2(V)
    b = 8.0 if mixed else 16.0
    alu, alu_name = (fp32_tflops, "fp32") if mixed else (fp64_tflops, "fp64")
    build_flops = V * (64.0 * 432 * c["diquarks"] + 24.0 * c["tensor_entries"] + 4.0 * c["row_terms"])
    work = {  # stage: (bytes, [(flops, peak TFLOP/s, pipe)])
        "ingest": (2 * 144 * V * (16.0 + b), []),
        "build": ((2 * 144 + c["block_rows"]) * V * b, [(build_flops, alu, alu_name)]),
        "fft_fwd": (2.0 * c["block_rows"] * V * b, [(5.0 * V * lg * c["block_rows"], alu, alu_name)]),
    }
    products = 8.0 * V * c["pair_macs"]
    sums = 4.0 * V * c["wick_terms"]
    if mixed and not stage_ms.get("wick"):
        work["contract"] = ((c["block_rows"] * b + c["outputs"] * 16.0) * V,
                            [(products, fp32_tflops, "fp32"), (sums, fp64_tflops, "fp64")])
    else:
        work["contract"] = ((c["block_rows"] + c["pair_items"]) * V * b,
                            [(products, fp32_tflops, "fp32") if mixed else (products, cmac_tflops, "fp64")])
        work["wick"] = ((c["pair_items"] * b + c["outputs"] * 16.0) * V, [(sums, fp64_tflops, "fp64")])
    work["fft_inv"] = (2.0 * c["outputs"] * V * 16.0, [(5.0 * V * lg * c["outputs"], alu, alu_name)])
    stages, floor = {}, 0.0
    for k, (nbytes, pipes) in work.items():
        times = [(nbytes * slices / (hbm * 1e9) * 1e3, "hbm")]
        times += [(flops * slices / (peak * 1e12) * 1e3, name) for flops, peak, name in pipes]
        f, bound = max(times)
        ms = stage_ms.get(k)
        stages[k] = {"floor_ms": f, "bound": bound, "ms": ms, "frac": f / ms if ms else None}
        floor += f
    return {"floor_ms": floor, "ms_per_step": step_ms, "frac": floor / step_ms, "hbm_gbs": hbm,
            "pipes_tflops": {"fp64": fp64_tflops, "fp64_cmac": cmac_tflops, "fp32": fp32_tflops},
            "counts": counts, "stages": stages}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="default workload: time the headline only (no legs, no CPU baseline), e.g. under a profiler")
    ap.add_argument("--workload", choices=["default", "config2", "batched", "L48", "decuplet"], default="default",
                    help="default: headline 48^3 x 96 (4 wall sources, 52 channels, complex64 propagators) in "
                         "FP64-accurate double-float arithmetic, with short legs (the same lattice in mixed "
                         "precision streamed from the host, the uneven batch, 16^3 x 32 in FP64 and double-float, "
                         "the 32^3 x 64 precision comparison); config2: 52 channels, 16^3 x 32, FP64 and mixed; "
                         "batched: 8 lattices, L in {16,24,32}, T in {32,48,64}, 4 sources each, mixed, one CUDA "
                         "graph per step; L48: 48^3 x 96, 4 sources, mixed, complex64 propagators streamed from "
                         "pinned host memory; decuplet: the 90 Omega Omega and p Omega ids, 16^3 x 32, FP64, "
                         "double-float and mixed")
    ap.add_argument("--error-report", action="store_true",
                    help="per-channel error of the mixed path against the FP64 path (L=32, T=64, t=32), "
                         "the FP64 path checked against the oracle at sampled points")
    ap.add_argument("--single-slice", choices=["fp64", "mixed", "bf16", "df64"], default=None,
                    help="run one time slice of the workload once and exit (small case for profilers)")
    ap.add_argument("--family", choices=["omega", "delta", "sigma", "xi"], default="omega",
                    help="--workload decuplet: the 90 Omega Omega and p Omega ids, the 90 Delta++ Delta++ and "
                         "p Delta++ ids, or the 81 Sigma*+ Sigma*+ or Xi*0 Xi*0 ids")
    ap.add_argument("--slice-L", type=int, default=None,
                    help="--single-slice on an L^3 x 2L lattice instead of 16^3 x 32")
    ap.add_argument("--slice-channels", default=None,
                    help="--single-slice on these comma-separated channel ids instead of the 52 (a smaller case "
                         "of the same kernels for profilers)")
    ap.add_argument("--tuning", default=None,
                    help="launch configuration for --single-slice: sites,threads,warps,chunk[,steps[,pair_groups]] "
                         "(as bbc_set_tuning)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(seed=0, n_points=1):
    """Time the CPU oracle on n_points (t, r) points of the workload, all 52
    channels and 16 spins each; returns (site*channels/s, seconds, cores)."""
    import synth
    import oracle.oracle as orc
    orc.build()
    L, T = L_BENCH, T_BENCH
    t = T // 2
    F = synth.flavour_set(L, T, 0, M_UD, M_S, seed=seed, times=[t])
    rng = np.random.default_rng(seed)
    r = list(rng.integers(0, L ** 3, size=n_points))
    t0 = time.perf_counter()
    orc.correlator(L, F["u"][0], F["d"][0], F["s"][0], list(range(N_CH)), r)
    dt = time.perf_counter() - t0
    cores = orc.threads()  # the OpenMP threads the oracle ran on
    return N_CH * n_points / dt, dt, cores


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n_pts = 16
    for _ in range(args.warmup):
        oracle_sample_L48(n_pts)
    secs = []
    for k in range(args.steps):
        v, dt, cores = oracle_sample_L48(n_pts)
        secs.append(dt)
    value = args.steps * n_pts / sum(secs)
    line = {
        "impl": "reference", "metric": "BB correlator site*channels/s", "value": value,
        "unit": "site*channels/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(secs) / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "all 52 channels, L=48, T=96, 4 wall sources (the headline lattice); each step the "
                               "CPU FP64 oracle (direct Wick sum over X) at 16 (r, channel) points: t=T/2, channel "
                               "p Xi- <- p Xi- (the cheapest octet channel), 16 random r, 16 spins each",
                   "L": L5, "T": T5, "sources": N_SRC5, "channels": N_CH},
        "cpu_baseline": {"value": value, "unit": "site*channels/s", "cores": cores, "kind": "oracle",
                         "sample": "per step: 48^3 lattice, t=T/2, p Xi- <- p Xi-, 16 random r, 16 spins, sums "
                                   "over all 110592 X"},
        "e2e": {"value": value, "unit": "site*channels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 8 and p[0].replace(".", "").isdigit():
                    rows.append(p)
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows]
        mx = max(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    try:
        run_ours(args, torch, rank, world, local)
    finally:
        if world > 1:
            torch.distributed.destroy_process_group()


def run_ours(args, torch, rank, world, local):
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import synth
    from paper_1510_00903_gb300 import build as _build
    _build.build()
    from paper_1510_00903_gb300 import bbc

    if args.error_report:
        return error_report(torch, dev, bbc, synth)
    if args.workload == "batched":
        return run_batched(args, torch, dev, bbc)
    if args.workload == "L48":
        return run_l48(args, torch, dev, bbc)
    if args.workload == "decuplet":
        return run_decuplet(args, torch, dev, bbc, synth)
    if args.workload == "default" and not args.single_slice:
        return run_default(args, torch, dev, bbc, synth)
    L, T = L_BENCH, T_BENCH
    V = L ** 3
    if args.single_slice:
        if args.slice_L:
            L, T = args.slice_L, 2 * args.slice_L
        chans = [int(x) for x in args.slice_channels.split(",")] if args.slice_channels else list(range(N_CH))
        t = T // 2
        F1 = synth.flavour_set(L, T, 0, M_UD, M_S, seed=1000, times=[t])
        prec = {"fp64": bbc.BBC_FP64, "mixed": bbc.BBC_MIXED_FP32, "bf16": bbc.BBC_MIXED_BF16,
                "df64": bbc.BBC_DF64}[args.single_slice]
        cor = bbc.Correlators(L, T, 0, M_UD, M_S, channels=chans, precision=prec, device=dev)
        if args.tuning:
            v = [int(x) for x in args.tuning.split(",")]
            cor.set_tuning({"build_sites": v[0], "build_threads": v[1], "fused_warps": v[2], "fused_chunk": v[3],
                            "fused_steps": v[4] if len(v) > 4 else 1, "pair_groups": v[5] if len(v) > 5 else 0})
        o = cor.run(torch.from_numpy(F1["u"]).to(dev), torch.from_numpy(F1["s"]).to(dev), [t])
        torch.cuda.synchronize(dev)
        print("single slice done", float(o.abs().max()))
        if prec == bbc.BBC_FP64:
            # the Sec. 2 projections of eight copies of the slice (436 MB, above the L2)
            R, Ra1 = cor.project(o.repeat(8, 1, 1, 1))
            torch.cuda.synchronize(dev)
            print("projection done", float(Ra1.abs().max()))
        cor.close()
        return
    from paper_1510_00903_gb300 import shard
    F = synth.flavour_set(L, T, 0, M_UD, M_S, **shard.rank_source(rank))
    Sl_h = torch.from_numpy(F["u"]).pin_memory()
    Ss_h = torch.from_numpy(F["s"]).pin_memory()
    Sl, Ss = Sl_h.to(dev), Ss_h.to(dev)
    chans = list(range(N_CH))
    stream = torch.cuda.current_stream(dev)
    out = torch.empty((T, N_CH, V, 16), dtype=torch.complex128, device=dev)

    def barrier():
        shard.barrier(world)

    def max_over_ranks(x):
        return shard.max_over_ranks(x, world, dev)

    def timed(cor, K, W, e2e=False, sampler=None):
        out_h = torch.empty(out.shape, dtype=out.dtype, pin_memory=True) if e2e else None
        src = (Sl_h, Ss_h) if e2e else (Sl, Ss)

        def step():
            if e2e:  # pinned host in and out, copies overlapped with the compute (the public streaming call)
                cor.run_to_host(src[0], src[1], range(T), out_h, normalised=True)
            else:
                cor.run(src[0], src[1], range(T), out=out, normalised=True)
        for _ in range(W):
            step()
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        bbc.bbc_enable_stage_timing(cor.ctx, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx_mgr = sampler if sampler else _Null()
        with ctx_mgr:
            e0.record(stream)
            for _ in range(K):
                step()
            e1.record(stream)
            torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / K
        stages = bbc.bbc_stage_timing(cor.ctx)
        bbc.bbc_enable_stage_timing(cor.ctx, False)
        return max_over_ranks(ms), stages

    # plain FP64 path (headline); launch shapes autotuned on slice 0 before timing
    cor = bbc.Correlators(L, T, 0, M_UD, M_S, channels=chans, precision=bbc.BBC_FP64, device=dev, stream=stream)
    sizes = cor.sizes()
    counts = plan_counts(bbc.bbc_plan_export(cor.ctx), sizes)
    tune_fp64, tune_fp64_ms = cor.autotune(Sl[0], Ss[0], t=0, reps=3)
    sampler = ClockSampler(local)
    ms, stages = timed(cor, args.steps, args.warmup, sampler=sampler)
    clocks = sampler.summary()
    ms_e2e, _ = timed(cor, max(1, args.steps // 2), 1, e2e=True)
    projection = measure_projection(torch, cor, out, stream)
    cor.close()
    value = shard.job_throughput(V * T * N_CH, world, ms)
    value_e2e = shard.job_throughput(V * T * N_CH, world, ms_e2e)

    # dominant kernel: the contraction (FP64 ALU bound)
    c_ms, c_n = stages["contract"]
    c_avg_ms = c_ms / max(c_n, 1)
    flops_per_launch = 8.0 * sizes["pair_macs_per_site"] * V
    achieved = flops_per_launch / (c_avg_ms * 1e-3) / 1e12
    here = os.path.dirname(os.path.abspath(__file__))
    traffic = profiled_traffic(os.path.join(here, "profiles", "k_pair_products_f64_L16_slice.md"),
                               os.path.join(here, "paper_1510_00903_gb300", "csrc", "pair_products.cu"),
                               sizes["pair_items"])
    roofline = {"bound": "alu", "kernel": "k_pair_products<double>", "achieved": achieved,
                "peak": FP64_CMAC_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_CMAC_PEAK_TFLOPS,
                "traffic": traffic, "peak_source": CMAC_PEAK_SOURCE,
                "algorithmic_flop_per_launch": flops_per_launch, "avg_launch_ms": c_avg_ms}
    stage_ms = {k: v[0] / args.steps for k, v in stages.items()}
    step_roof = step_roofline(counts, V, T, stage_ms, ms)

    def mixed_leg(precision, note, components=bbc.BBC_UPPER):
        corm = bbc.Correlators(L, T, 0, M_UD, M_S, channels=chans, precision=precision, device=dev, stream=stream,
                               components=components)
        tune_m, tune_m_ms = corm.autotune(Sl[0], Ss[0], t=0, reps=3)
        ms_m, st_m = timed(corm, args.steps, args.warmup)
        corm.close()
        cm_ms, cm_n = st_m["contract"]
        cm_avg = cm_ms / max(cm_n, 1)
        stage_m = {k: v[0] / args.steps for k, v in st_m.items()}
        leg = {"value": shard.job_throughput(V * T * N_CH, world, ms_m), "ms_per_step": ms_m,
               "speedup_vs_fp64": ms / ms_m, "precision": note, "stage_ms_per_step": stage_m,
               "contract_tflops": flops_per_launch / (cm_avg * 1e-3) / 1e12,
               "contract_frac_fp32_peak": flops_per_launch / (cm_avg * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
               "tuning": tune_m, "autotune_ms": tune_m_ms}
        if precision == bbc.BBC_MIXED_FP32 and components == bbc.BBC_UPPER:
            leg["step_roofline"] = step_roofline(counts, V, T, stage_m, ms_m, mixed=True)
        return leg

    # FP64 with double-float block-pair products (FP64-accurate, FP32 pipes)
    cord = bbc.Correlators(L, T, 0, M_UD, M_S, channels=chans, precision=bbc.BBC_DF64, device=dev, stream=stream)
    tune_d, _ = cord.autotune(Sl[0], Ss[0], t=0, reps=3)
    ms_d, st_d = timed(cord, args.steps, args.warmup)
    cord.close()
    cd_ms, cd_n = st_d["contract"]
    df64 = {"value": shard.job_throughput(V * T * N_CH, world, ms_d), "ms_per_step": ms_d, "speedup_vs_fp64": ms / ms_d,
            "precision": "propagators, block build, FFTs, block-pair products and Wick sums in double-float "
                         "arithmetic (two FP32 words, 48-bit significand) on the FP32 pipes; FP64 for the input split "
                         "and the normalisation; parity-tested against the FP64 oracle at 1e-12",
            "stage_ms_per_step": {k: v[0] / args.steps for k, v in st_d.items()},
            "contract_ms_per_slice": cd_ms / max(cd_n, 1), "tuning": tune_d}

    mixed = bf16 = lower = None
    if not args.no_mixed:
        lower = mixed_leg(bbc.BBC_MIXED_FP32, "lower Dirac components (antibaryons backward in time), mixed FP32",
                          components=bbc.BBC_LOWER)
        mixed = mixed_leg(bbc.BBC_MIXED_FP32, "FP32 blocks, FFTs and products (tensor-core split-TF32 products "
                                              "for the trace-form pairs); double-float Wick sums, FP64 "
                                              "normalisation (per-channel errors: --error-report)")
        bf16 = mixed_leg(bbc.BBC_MIXED_BF16, "trial: Fourier-space blocks rounded to bfloat16 before the FP32 "
                                             "products (per-channel errors: --error-report)")

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, dt, cores = oracle_sample(seed=7)
        cpu = {"value": v, "unit": "site*channels/s", "cores": cores, "kind": "oracle",
               "sample": f"t=T/2, one random r, all 52 channels x 16 spins, sum over all {V} X ({dt:.1f} s)"}
    cnt = {"load": 2, "build": 4, "contract": 6}
    launches = args.steps * T * (2 * cnt["load"] + cnt["build"] + cnt["contract"])
    line = {
        "metric": "BB correlator site*channels/s", "value": value, "unit": "site*channels/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_SITE_CH_PER_S,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "all 52 channels, L=16, T=32, one wall source, complex128 propagators, plain FP64",
                   "L": L, "T": T, "channels": N_CH, "precision": "fp64",
                   "l2": f"no flush: block fields of one slice ({V * sizes['block_outputs'] * 16 / 1e6:.0f} MB) "
                         "exceed the 129 MB L2"},
        "e2e": {"value": value_e2e, "unit": "site*channels/s",
                "h2d_bytes_per_step": int(2 * T * V * 144 * 16),
                "d2h_bytes_per_step": int(out.numel() * 16)},
        "gpu_launches": launches,
        "roofline": roofline,
        "stage_ms_per_step": stage_ms,
        "step_roofline": step_roof,
        # the paper's split of a step (Sec. 5, Table ElapsedTime): Step-1 = blocks
        # and forward FFT, Step-2 = contraction and inverse FFT (best 32-node BG/Q
        # split: 6 s + 13 s)
        "paper_steps_ms": {"step1": stage_ms.get("ingest", 0) + stage_ms.get("build", 0) + stage_ms.get("fft_fwd", 0),
                           "step2": stage_ms.get("contract", 0) + stage_ms.get("wick", 0) + stage_ms.get("fft_inv", 0)
                           + stage_ms.get("normalise", 0),
                           "paper_best_bgq_s": {"step1": 6, "step2": 13}},
        "plan": sizes,
        "tuning": {"chosen": tune_fp64, "autotune_ms": tune_fp64_ms},
        "df64": df64,
        "mixed": mixed,
        "bf16_trial": bf16,
        "lower_components": lower,
        "projection": projection,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def measure_projection(torch, cor, C, stream, reps=20):
    """Spin-state and cubic-group projections (Sec. 2) of the correlators of
    every slice of one step (one launch over T x 52 fields): an epilogue
    outside the timed step, timed on its own.  Algorithmic bytes: C read
    once, R and Ra1 written once."""
    R, Ra1 = torch.empty_like(C), torch.empty_like(C)
    for _ in range(3):
        cor.project(C, R, Ra1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        cor.project(C, R, Ra1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nbytes = 3 * C.numel() * 16
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"kernel": "k_project", "bound": "hbm", "ms_per_launch": ms, "fields": C.numel() // (C.shape[-2] * 16),
            "algorithmic_bytes": nbytes, "achieved_gbs": gbs, "peak_gbs": HBM_PEAK_GBS,
            "peak_source": HBM_PEAK_SOURCE, "frac": gbs / HBM_PEAK_GBS, "l2": "C, R, Ra1 of all slices (3 x 1.74 GB) exceed the L2"}


def error_report(torch, dev, bbc, synth, reps=3):
    """Per-channel max |mixed - fp64| / max |fp64| over r and spin on one slice
    of the L=32, T=64 workload; the FP64 result against the oracle at r = 0
    and two random r for four channels; and the time of that slice in each
    precision (launch shapes autotuned on it, device-resident inputs, CUDA
    events over `reps` runs after one untimed run)."""
    import oracle.oracle as orc
    L, T, t = 32, 64, 32
    F = synth.flavour_set(L, T, 0, M_UD, M_S, seed=3, times=[t])
    Sl, Ss = torch.from_numpy(F["u"]).to(dev), torch.from_numpy(F["s"]).to(dev)
    res, ms = {}, {}
    stream = torch.cuda.current_stream(dev)
    for name, prec in (("fp64", bbc.BBC_FP64), ("df64", bbc.BBC_DF64), ("mixed", bbc.BBC_MIXED_FP32),
                       ("bf16", bbc.BBC_MIXED_BF16)):
        cor = bbc.Correlators(L, T, 0, M_UD, M_S, channels=list(range(N_CH)), precision=prec, device=dev,
                              stream=stream)
        cor.autotune(Sl[0], Ss[0], t=t, reps=2)
        out = cor.run(Sl, Ss, [t], normalised=True)
        res[name] = out[0].cpu().numpy()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(reps):
            cor.run(Sl, Ss, [t], out=out, normalised=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms[name] = e0.elapsed_time(e1) / reps
        cor.close()
    a, b = res["mixed"], res["fp64"]
    scale = np.abs(b).reshape(N_CH, -1).max(axis=1)
    err = np.abs(a - b).reshape(N_CH, -1).max(axis=1) / scale
    err16 = np.abs(res["bf16"] - b).reshape(N_CH, -1).max(axis=1) / scale
    chans, r_list = [0, 10, 41, 51], [0, 12345, 30001]
    want = orc.normalise(orc.correlator(L, F["u"][0], F["d"][0], F["s"][0], chans, r_list), chans, t, M_UD, M_S)
    o_err = float((np.abs(b[chans][:, r_list] - want).reshape(len(chans), -1).max(axis=1) / scale[chans]).max())
    errdf = np.abs(res["df64"] - b).reshape(N_CH, -1).max(axis=1) / scale
    print(json.dumps({"report": "mixed precision error per channel", "L": L, "T": T, "t": t,
                      "metric": "max_{r,s}|C_mixed - C_fp64| / max_{r,s}|C_fp64|",
                      "per_channel": [float(x) for x in err], "max": float(err.max()), "median": float(np.median(err)),
                      "bf16_per_channel": [float(x) for x in err16], "bf16_max": float(err16.max()),
                      "bf16_median": float(np.median(err16)), "df64_max": float(errdf.max()),
                      "fp64_vs_oracle_sampled": o_err,
                      "ms_per_slice": ms, "site_channels_per_s": {k: L ** 3 * N_CH / (v * 1e-3) for k, v in ms.items()},
                      "speedup_vs_fp64": {k: ms["fp64"] / v for k, v in ms.items()}}), flush=True)


def device_propagators(torch, dev, L, T, t0, mass, seed):
    """Synthetic propagators generated on the device (complex64, Re and Im
    ~ N(0, 1/2), times exp(-mass ((t - t0) mod T))) for throughput runs too
    large to draw on the host."""
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    d = ((torch.arange(T, device=dev) - t0) % T).to(torch.float32)
    S = torch.randn((T, L ** 3, 144), dtype=torch.complex64, device=dev, generator=g)
    return (S * torch.exp(-mass * d)[:, None, None]).view(T, L ** 3, 12, 12)


def emit(line):
    print(json.dumps(line), flush=True)


def run_batched(args, torch, dev, bbc):
    lattices = [(16, 32), (16, 48), (24, 32), (24, 48), (24, 64), (32, 48), (32, 64), (16, 64)]
    from paper_1510_00903_gb300 import shard
    rank, world, _ = dist_env()
    sd = 1000 * rank  # every rank its own gauge configurations (independent units)
    inputs = [(device_propagators(torch, dev, L, T, 0, M_UD, sd + 10 + i),
               device_propagators(torch, dev, L, T, 0, M_S, sd + 50 + i))
              for i, (L, T) in enumerate(lattices)]
    b = bbc.LatticeBatch(lattices, inputs, n_sources=4, channels=list(range(N_CH)), precision=bbc.BBC_MIXED_FP32,
                         device=dev)
    tuned = b.autotune()
    t_cap = time.perf_counter()
    g = b.capture()
    t_cap = time.perf_counter() - t_cap
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize(dev)
    shard.barrier(world)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(dev.index)
    with sampler:
        e0.record(b.stream)
        for _ in range(args.steps):
            g.replay()
        e1.record(b.stream)
        torch.cuda.synchronize(dev)
    shard.barrier(world)
    torch.cuda.synchronize(dev)
    ms = shard.max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    units = b.sites_channels()
    slices = sum(4 * T for _, T in lattices)
    b.close()
    if rank != 0:
        return
    emit({"metric": "BB correlator site*channels/s", "value": shard.job_throughput(units, world, ms),
          "unit": "site*channels/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
          "config": {"workload": "batched: 8 lattices (L,T) in " + str(lattices) + ", 4 wall sources each "
                     "(t0 = 0, T/4, T/2, 3T/4), 52 channels, mixed precision, complex64 propagators, "
                     "one CUDA graph per step", "slices_per_step": slices,
                     "l2": "no flush: block fields of one slice (>= 241 MB) exceed the 129 MB L2"},
          "graph": {"capture_s": t_cap, "launches_per_step": 1}, "tuning": {str(k): v for k, v in tuned.items()},
          "clocks": sampler.summary()})


def run_decuplet(args, torch, dev, bbc, synth):
    """The decuplet channels of the Sec. 4 footnote: all 81 Omega_l1 Omega_l2 <-
    Omega_l3 Omega_l4 and 9 p Omega_l <- p Omega_l' ids in one context, 16^3 x 32,
    one wall source, device-resident complex128 propagators; FP64 (headline),
    double-float and mixed FP32 (fused: this list's rows and products fit
    one CTA's shared memory)."""
    from paper_1510_00903_gb300 import shard
    rank, world, _ = dist_env()
    L, T = L_BENCH, T_BENCH
    V = L ** 3
    chans, label = {"omega": (bbc.OMEGA_OMEGA + bbc.P_OMEGA, "90 decuplet channels (81 Omega Omega, 9 p Omega)"),
                    "delta": (bbc.DELTA_DELTA + bbc.P_DELTA, "90 decuplet channels (81 Delta++ Delta++, 9 p Delta++)"),
                    "sigma": (bbc.SIGMA_STAR_PAIRS, "81 decuplet channels (Sigma*+ Sigma*+)"),
                    "xi": (bbc.XI_STAR_PAIRS, "81 decuplet channels (Xi*0 Xi*0)")}[args.family]
    F = synth.flavour_set(L, T, 0, M_UD, M_S, **shard.rank_source(rank))
    Sl, Ss = torch.from_numpy(F["u"]).to(dev), torch.from_numpy(F["s"]).to(dev)
    stream = torch.cuda.current_stream(dev)
    out = torch.empty((T, len(chans), V, 16), dtype=torch.complex128, device=dev)
    legs = {}
    sizes = None
    clocks = None
    for name, prec in (("fp64", bbc.BBC_FP64), ("df64", bbc.BBC_DF64), ("mixed", bbc.BBC_MIXED_FP32)):
        cor = bbc.Correlators(L, T, 0, M_UD, M_S, channels=chans, precision=prec, device=dev, stream=stream)
        sizes = cor.sizes()
        counts = plan_counts(bbc.bbc_plan_export(cor.ctx), sizes)
        tune, _ = cor.autotune(Sl[0], Ss[0], t=0, reps=2)
        for _ in range(args.warmup):
            cor.run(Sl, Ss, range(T), out=out, normalised=True)
        torch.cuda.synchronize(dev)
        shard.barrier(world)
        torch.cuda.synchronize(dev)
        bbc.bbc_enable_stage_timing(cor.ctx, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(dev.index) if name == "fp64" else _Null()
        with sampler:
            e0.record(stream)
            for _ in range(args.steps):
                cor.run(Sl, Ss, range(T), out=out, normalised=True)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        shard.barrier(world)
        torch.cuda.synchronize(dev)
        if name == "fp64":
            clocks = sampler.summary()
        stages = bbc.bbc_stage_timing(cor.ctx)
        cor.close()
        ms = shard.max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
        c_ms, c_n = stages["contract"]
        flop = 8.0 * sizes["pair_macs_per_site"] * V
        stage_ms = {k: v[0] / args.steps for k, v in stages.items()}
        legs[name] = {"value": shard.job_throughput(V * T * len(chans), world, ms), "ms_per_step": ms,
                      "stage_ms_per_step": stage_ms,
                      "contract_ms_per_slice": c_ms / max(c_n, 1),
                      "contract_tflops": flop / (c_ms / max(c_n, 1) * 1e-3) / 1e12, "tuning": tune}
        if name != "df64":  # double-float arithmetic has no pipe peak of its own
            legs[name]["step_roofline"] = step_roofline(counts, V, T, stage_ms, ms, mixed=name == "mixed")
    if rank != 0:
        return
    fp = legs["fp64"]
    emit({"metric": "BB correlator site*channels/s", "value": fp["value"], "unit": "site*channels/s",
          "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": fp["ms_per_step"],
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": {"workload": label + ", L=16, T=32, one wall source, complex128 propagators, plain FP64",
                     "L": L, "T": T, "channels": len(chans),
                     "l2": f"no flush: block fields of one slice ({V * sizes['block_outputs'] * 16 / 1e6:.0f} MB) "
                           "exceed the 129 MB L2"},
          "roofline": {"bound": "alu", "kernel": "k_pair_products<double>", "achieved": fp["contract_tflops"],
                       "peak": FP64_CMAC_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": fp["contract_tflops"] / FP64_CMAC_PEAK_TFLOPS, "traffic": None,
                       "peak_source": CMAC_PEAK_SOURCE},
          "plan": sizes, "fp64": fp, "df64": legs["df64"], "mixed": legs["mixed"], "clocks": clocks})


def run_l48(args, torch, dev, bbc):
    """48^3 x 96, 4 wall sources, mixed precision; the complex64 propagators of
    every slice go host -> device inside the step (streamed per slice)."""
    from paper_1510_00903_gb300 import shard
    rank, world, _ = dist_env()
    L, T, n_src = 48, 96, 4
    S_dev = [device_propagators(torch, dev, L, T, 0, m, 1000 * rank + s) for m, s in ((M_UD, 91), (M_S, 92))]
    S_host = [x.cpu().pin_memory() for x in S_dev]
    del S_dev
    cors = []
    ws = None
    stream = torch.cuda.Stream(dev)
    for k in range(n_src):
        c = bbc.Correlators(L, T, (k * T) // n_src, M_UD, M_S, channels=list(range(N_CH)),
                            precision=bbc.BBC_MIXED_FP32, device=dev, stream=stream, workspace=ws)
        ws = c.workspace
        cors.append(c)
    with torch.cuda.stream(stream):
        tuned, _ = cors[0].autotune(S_host[0][0], S_host[1][0], t=0, reps=2)
    for c in cors[1:]:
        c.set_tuning(tuned)
    out = torch.empty((N_CH, L ** 3, 16), dtype=torch.complex128, device=dev)

    def step():
        # host -> device copy of slice t+1 overlapped with the compute of slice t
        with torch.cuda.stream(stream):
            for c in cors:
                c.run_streamed(S_host[0], S_host[1], range(T), out)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    shard.barrier(world)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(dev.index)
    with sampler:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    shard.barrier(world)
    torch.cuda.synchronize(dev)
    ms = shard.max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    units = n_src * T * L ** 3 * N_CH
    for c in cors:
        c.close()
    if rank != 0:
        return
    emit({"metric": "BB correlator site*channels/s", "value": shard.job_throughput(units, world, ms),
          "unit": "site*channels/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
          "config": {"workload": "52 channels, L=48, T=96, 4 wall sources, mixed precision, complex64 propagators "
                     "streamed host->device per slice inside the step (copy of slice t+1 overlapped with slice t)", "h2d_bytes_per_step": int(
                         n_src * T * 2 * L ** 3 * 144 * 8),
                     "l2": "no flush: block fields of one slice (6.5 GB) exceed the 129 MB L2"},
          "tuning": tuned, "clocks": sampler.summary()})


# ------------------------------------------------------------ default run
#: headline lattice: 48^3 x 96, four wall sources, 52 channels, complex64 storage
L5, T5, N_SRC5 = 48, 96, 4
#: slices per headline step: a quarter of one source's time slices, so 16
#: steps cover the four sources once and 20 timed steps stay near a minute
HEAD_SLICES = 24
#: double-float arithmetic on the FP32 pipes: one complex multiply-add of the
#: block-pair products is four double-float multiply-adds of 12 FP32
#: instructions each (TwoProduct of the high words, the cross terms, TwoSum
#: into the accumulator)
DF_INSTR_PER_CMAC = 48
#: FP32 instruction issue of the whole GPU: 152 SMs x 128 lanes x 2070 MHz
FP32_ISSUE_TOPS = 152 * 128 * 2.070e9 / 1e12
DF_CMAC_PEAK_TFLOPS = FP32_ISSUE_TOPS / DF_INSTR_PER_CMAC * 8.0
DF_PEAK_SOURCE = "derived: 40.27 T FP32 instr/s / 48 instr per double-float complex MAC x 8 flop"


def channel_errors(torch, got, ref):
    """Per channel: max over r and spin of |got - ref| / max |ref| (device tensors [n_ch, V, 16]);
    returns the maximum and median over channels and the worst channel."""
    num = (got - ref).abs().flatten(1).amax(dim=1)
    den = ref.abs().flatten(1).amax(dim=1)
    e = (num / den).double().cpu().numpy()
    return {"max": float("%.3g" % e.max()), "median": float("%.3g" % np.median(e)), "worst_channel": int(e.argmax())}


def timed_steps(torch, dev, stream, step, K, W, world, sampler=None):
    """W untimed then K timed calls of step(k) between barriers; CUDA events on `stream`."""
    from paper_1510_00903_gb300 import shard
    for k in range(W):
        step(k)
    torch.cuda.synchronize(dev)
    shard.barrier(world)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with (sampler if sampler else _Null()):
        e0.record(stream)
        for k in range(K):
            step(W + k)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    shard.barrier(world)
    torch.cuda.synchronize(dev)
    return shard.max_over_ranks(e0.elapsed_time(e1) / K, world, dev)


def oracle_sample_L48(n_points):
    """The oracle on the headline lattice: one channel (p Xi- <- p Xi-, the
    cheapest octet channel), n_points random r at t = T/2, each a sum over all
    48^3 X (sink tensors included); returns (site*channels/s, seconds, cores)."""
    import synth
    import oracle.oracle as orc
    orc.build()
    t = T5 // 2
    F = synth.flavour_set(L5, T5, 0, M_UD, M_S, seed=5, times=[t])
    rng = np.random.default_rng(t)
    r = list(rng.integers(0, L5 ** 3, size=n_points))
    t0 = time.perf_counter()
    orc.correlator(L5, F["u"][0], F["d"][0], F["s"][0], [16], r)
    dt = time.perf_counter() - t0
    return n_points / dt, dt, min(n_points, orc.threads())


def run_default(args, torch, dev, bbc, synth):
    """Headline: 48^3 x 96, 4 wall sources, 52 channels, complex64 propagators,
    FP64-accurate double-float arithmetic, inputs resident in HBM; e2e the same
    through Correlators.run_to_host (pinned host in and out).  Legs: the same
    lattice in mixed precision streamed from pinned host memory, the uneven
    batch as one CUDA graph, 16^3 x 32 in FP64 and double-float, the
    precision comparison on one 32^3 x 64 slice; each leg's error is measured
    against the FP64 path on one slice."""
    from paper_1510_00903_gb300 import shard
    rank, world, local = dist_env()
    chans = list(range(N_CH))
    V5 = L5 ** 3
    here = os.path.dirname(os.path.abspath(__file__))
    stream = torch.cuda.Stream(dev)
    # one source's wall-source propagators (complex64); the four sources share the draw
    S_dev = [device_propagators(torch, dev, L5, T5, 0, m, 1000 * rank + s) for m, s in ((M_UD, 91), (M_S, 92))]
    torch.cuda.synchronize(dev)
    out = torch.empty((N_CH, V5, 16), dtype=torch.complex128, device=dev)

    # ---- headline: double-float, HEAD_SLICES slices of one source per step
    cors, ws = [], None
    for k in range(N_SRC5):
        c = bbc.Correlators(L5, T5, (k * T5) // N_SRC5, M_UD, M_S, channels=chans, precision=bbc.BBC_DF64,
                            device=dev, stream=stream, workspace=ws)
        ws = c.workspace
        cors.append(c)
    sizes = cors[0].sizes()
    tune, _ = cors[0].autotune(S_dev[0][0], S_dev[1][0], t=0, reps=1)
    for c in cors[1:]:
        c.set_tuning(tune)
    def head_step(k):
        src, part = (k // 4) % N_SRC5, k % 4
        cors[src].run_each(S_dev[0], S_dev[1], range(HEAD_SLICES * part, HEAD_SLICES * (part + 1)), out)

    bbc.bbc_enable_stage_timing(cors[0].ctx, True)
    for c in cors[1:]:
        bbc.bbc_enable_stage_timing(c.ctx, True)
    sampler = ClockSampler(local)
    ms = timed_steps(torch, dev, stream, head_step, args.steps, args.warmup, world, sampler)
    clocks = sampler.summary()
    stage_tot = {}
    n_contract = 0
    for c in cors:
        st = bbc.bbc_stage_timing(c.ctx)
        for key, (v, n) in st.items():
            stage_tot[key] = stage_tot.get(key, 0.0) + v
        n_contract += st["contract"][1]
        bbc.bbc_enable_stage_timing(c.ctx, False)
    # timing covered warm-up and timed steps: the per-step stage times are averages over both
    n_steps_timed = args.steps + args.warmup
    stage_ms = {k: v / n_steps_timed for k, v in stage_tot.items()}
    c_avg = stage_tot["contract"] / max(n_contract, 1)
    flop = 8.0 * sizes["pair_macs_per_site"] * V5
    achieved = flop / (c_avg * 1e-3) / 1e12
    # DRAM bytes per launch from the ncu capture of the 16^3 slice (the full-size
    # launch is too large to capture), scaled to 48^3 by the sites processed
    traffic16 = profiled_traffic(os.path.join(here, "profiles", "k_pair_products_df_L16_slice.md"),
                                 os.path.join(here, "paper_1510_00903_gb300", "csrc", "pair_products_df.cu"),
                                 sizes["pair_items"])
    traffic = None if traffic16 is None else traffic16 * V5 / L_BENCH ** 3
    value = shard.job_throughput(HEAD_SLICES * V5 * N_CH, world, ms)
    # e2e: pinned host propagators in, pinned host correlators out (two-slice ring)
    S_host = [x[:HEAD_SLICES].cpu().pin_memory() for x in S_dev]
    ring = torch.empty((2, N_CH, V5, 16), dtype=torch.complex128, pin_memory=True)

    def e2e_step(k):
        cors[k % N_SRC5].run_to_host(S_host[0], S_host[1], range(HEAD_SLICES), ring)

    k_e2e = max(1, args.steps // 4)
    ms_e2e = timed_steps(torch, dev, stream, e2e_step, k_e2e, 1, world)
    del S_host, ring
    # error of one slice against the FP64 path on the same inputs
    t_chk = 50
    cors[0].run_each(S_dev[0], S_dev[1], [t_chk], out)
    ref64 = bbc.Correlators(L5, T5, 0, M_UD, M_S, channels=chans, precision=bbc.BBC_FP64, device=dev, stream=stream)
    ref_out = torch.empty_like(out)
    ref64.run_each(S_dev[0], S_dev[1], [t_chk], ref_out)
    torch.cuda.synchronize(dev)
    head_err = channel_errors(torch, out, ref_out)
    for c in cors:
        c.close()
    del cors, ws

    if args.headline_only:
        ref64.close()
        if rank == 0:
            print(json.dumps({"metric": "BB correlator site*channels/s", "value": value, "ms_per_step": ms,
                              "roofline_achieved": achieved, "err_vs_fp64": head_err,
                              "stage_ms_per_step": stage_ms}), flush=True)
        return
    # ---- leg: the same lattice, mixed precision (tensor cores), streamed from pinned host memory
    mcors, mws = [], None
    for k in range(N_SRC5):
        c = bbc.Correlators(L5, T5, (k * T5) // N_SRC5, M_UD, M_S, channels=chans, precision=bbc.BBC_MIXED_FP32,
                            device=dev, stream=stream, workspace=mws)
        mws = c.workspace
        mcors.append(c)
    S_host_all = [x.cpu().pin_memory() for x in S_dev]
    mtune, _ = mcors[0].autotune(S_dev[0][0], S_dev[1][0], t=0, reps=1)
    for c in mcors[1:]:
        c.set_tuning(mtune)
    bbc.bbc_enable_stage_timing(mcors[0].ctx, True)

    def mixed_step(k):
        mcors[k % N_SRC5].run_streamed(S_host_all[0], S_host_all[1], range(T5), out)

    k_leg = max(2, min(3, args.steps))
    ms_mixed = timed_steps(torch, dev, stream, mixed_step, k_leg, 1, world)
    st_m = bbc.bbc_stage_timing(mcors[0].ctx)
    mcors[0].run_each(S_dev[0], S_dev[1], [t_chk], out)
    torch.cuda.synchronize(dev)
    mixed_err = channel_errors(torch, out, ref_out)
    mcounts = plan_counts(bbc.bbc_plan_export(mcors[0].ctx), mcors[0].sizes())
    n_m = max(st_m["build"][1], 1)
    mstage = {k: v[0] / n_m * T5 for k, v in st_m.items()}  # per source of 96 slices
    mixed_roof = step_roofline(mcounts, V5, T5, mstage, ms_mixed, mixed=True)
    for c in mcors:
        c.close()
    ref64.close()
    del mcors, mws, S_host_all, ref64, ref_out, S_dev, out

    # ---- leg: 16^3 x 32 in FP64 and double-float (the paper's lattice), inputs in HBM
    L2_, T2_ = L_BENCH, T_BENCH
    V2 = L2_ ** 3
    F2 = synth.flavour_set(L2_, T2_, 0, M_UD, M_S, **shard.rank_source(rank))
    S2 = [torch.from_numpy(F2["u"]).to(dev), torch.from_numpy(F2["s"]).to(dev)]
    out2 = torch.empty((T2_, N_CH, V2, 16), dtype=torch.complex128, device=dev)
    legs16 = {}
    ref16 = None
    for name, prec in (("fp64", bbc.BBC_FP64), ("df64", bbc.BBC_DF64), ("mixed", bbc.BBC_MIXED_FP32),
                       ("tf32_trial", bbc.BBC_MIXED_TF32)):
        c = bbc.Correlators(L2_, T2_, 0, M_UD, M_S, channels=chans, precision=prec, device=dev, stream=stream)
        sz = c.sizes()
        cnt = plan_counts(bbc.bbc_plan_export(c.ctx), sz)
        tn, _ = c.autotune(S2[0][0], S2[1][0], t=0, reps=2)
        bbc.bbc_enable_stage_timing(c.ctx, True)
        k16 = max(2, min(5, args.steps))
        m16 = timed_steps(torch, dev, stream, lambda k: c.run(S2[0], S2[1], range(T2_), out=out2), k16, 2, world)
        st16 = bbc.bbc_stage_timing(c.ctx)
        sm16 = {k: v[0] / (k16 + 2) for k, v in st16.items()}
        leg = {"value": shard.job_throughput(V2 * T2_ * N_CH, world, m16), "ms_per_step": round(m16, 3)}
        if name == "fp64":
            ref16 = out2[16].clone()
            ca = st16["contract"][0] / max(st16["contract"][1], 1)
            ach = 8.0 * sz["pair_macs_per_site"] * V2 / (ca * 1e-3) / 1e12
            leg["roofline"] = {"kernel": "k_pair_products<double>", "achieved": round(ach, 4),
                               "peak": FP64_CMAC_PEAK_TFLOPS, "frac": round(ach / FP64_CMAC_PEAK_TFLOPS, 4),
                               "traffic": profiled_traffic(
                                   os.path.join(here, "profiles", "k_pair_products_f64_L16_slice.md"),
                                   os.path.join(here, "paper_1510_00903_gb300", "csrc", "pair_products.cu"),
                                   sz["pair_items"])}
        else:
            leg["err_vs_fp64"] = channel_errors(torch, out2[16], ref16)
        if prec in (bbc.BBC_FP64, bbc.BBC_MIXED_FP32):
            roof = step_roofline(cnt, V2, T2_, sm16, m16, mixed=prec == bbc.BBC_MIXED_FP32)
            leg["step_roofline"] = {"floor_ms": round(roof["floor_ms"], 3), "frac": round(roof["frac"], 4)}
            leg["stage_ms"] = {k: round(v, 2) for k, v in sm16.items() if v}
        if name == "fp64":
            pj = measure_projection(torch, c, out2, stream)
            leg["projection"] = {"ms": round(pj["ms_per_launch"], 3), "gbs": round(pj["achieved_gbs"], 1),
                                 "frac": round(pj["frac"], 4)}
        legs16[name] = leg
        c.close()
    del out2, S2

    # ---- leg: the uneven batch (8 lattices x 4 sources, mixed, complex64) as one CUDA graph per step
    batched = batched_leg(args, torch, dev, bbc, world)

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, dt, cores = oracle_sample_L48(16)
        cpu = {"value": v, "unit": "site*channels/s", "cores": cores, "kind": "oracle",
               "sample": f"48^3, t=T/2, p Xi- <- p Xi- (cheapest channel), 16 random r x 16 spins, all X ({dt:.1f} s)"}
    c0 = bbc.bbc_create(L5, T5, 0, M_UD, M_S, bbc.BBC_DF64, chans)
    lc = bbc.bbc_launch_counts(c0)
    bbc.bbc_destroy(c0)
    launches = args.steps * HEAD_SLICES * (2 * lc["load"] + lc["build"] + lc["contract"])
    line = {
        "metric": "BB correlator site*channels/s", "value": value, "unit": "site*channels/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "df64", "data": "synthetic",
        "config": {"workload": "52 channels, L=48, T=96, 4 wall sources (one shared synthetic draw), complex64 "
                               "propagators in HBM, FP64-accurate double-float arithmetic; a step is "
                               f"{HEAD_SLICES} slices of one source (16 steps = the 4 sources)",
                   "L": L5, "T": T5, "sources": N_SRC5, "channels": N_CH, "slices_per_step": HEAD_SLICES,
                   "l2": "no flush: one slice's blocks (13 GB) exceed the 129 MB L2"},
        "e2e": {"value": shard.job_throughput(HEAD_SLICES * V5 * N_CH, world, ms_e2e), "unit": "site*channels/s",
                "h2d_bytes_per_step": int(HEAD_SLICES * 2 * V5 * 144 * 8),
                "d2h_bytes_per_step": int(HEAD_SLICES * N_CH * V5 * 16 * 16)},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": "k_pair_products_df", "achieved": achieved, "peak": DF_CMAC_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / DF_CMAC_PEAK_TFLOPS, "traffic": traffic,
                     "peak_source": DF_PEAK_SOURCE, "avg_launch_ms": round(c_avg, 3)},
        "err_vs_fp64": head_err,
        "stage_ms_per_step": {k: round(v, 1) for k, v in stage_ms.items() if v > 0.5},
        # legs, one array each: [site*channels/s, ms per step, step roofline frac, max per-channel error vs FP64]
        "legs": {
            "fields": ["value", "ms_per_step", "step_roofline_frac", "err_vs_fp64_max"],
            "mixed_L48_streamed": [shard.job_throughput(T5 * V5 * N_CH, world, ms_mixed), round(ms_mixed, 1),
                                   round(mixed_roof["frac"], 3), mixed_err["max"]],
            "batched_config4": [batched["value"], batched["ms_per_step"], None, batched["err_vs_fp64"]["max"]],
        },
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    for name, leg in legs16.items():
        line["legs"][name + "_L16"] = [leg["value"], leg["ms_per_step"], leg.get("step_roofline", {}).get("frac"),
                                       leg.get("err_vs_fp64", {}).get("max")]
    line["legs"]["fp64_L16_kernel_roofline"] = legs16["fp64"]["roofline"]
    line["legs"]["projection_L16"] = legs16["fp64"]["projection"]
    # the legs in full (stage times, floors, errors), one line before the result line
    detail = {"detail": "legs of the line below", "mixed_L48_streamed": {
        "value": shard.job_throughput(T5 * V5 * N_CH, world, ms_mixed), "ms_per_step": ms_mixed,
        "slices_per_step": T5, "step_roofline": {"floor_ms": mixed_roof["floor_ms"], "frac": mixed_roof["frac"]},
        "err_vs_fp64": mixed_err, "stage_ms": {k: round(v, 1) for k, v in mstage.items() if v > 0.5}},
        "L16_T32": legs16, "batched": batched, "headline_tuning": tune}
    print(json.dumps(detail), flush=True)
    print(json.dumps(line), flush=True)


def batched_leg(args, torch, dev, bbc, world):
    """The uneven batch (8 lattices, 4 sources each, 52 channels, mixed,
    complex64) recorded as one CUDA graph; a step is one replay.  Error: one
    L=32 slice of the batch against the FP64 path."""
    lattices = [(16, 32), (16, 48), (24, 32), (24, 48), (24, 64), (32, 48), (32, 64), (16, 64)]
    rank = dist_env()[0]
    sd = 1000 * rank
    inputs = [(device_propagators(torch, dev, L, T, 0, M_UD, sd + 10 + i),
               device_propagators(torch, dev, L, T, 0, M_S, sd + 50 + i))
              for i, (L, T) in enumerate(lattices)]
    b = bbc.LatticeBatch(lattices, inputs, n_sources=4, channels=list(range(N_CH)), precision=bbc.BBC_MIXED_FP32,
                         device=dev)
    tuned = b.autotune(reps=1)
    t_cap = time.perf_counter()
    g = b.capture()
    t_cap = time.perf_counter() - t_cap
    ms = timed_steps(torch, dev, b.stream, lambda k: g.replay(), max(2, min(3, args.steps)), 1, world)
    # error: slice 40 of the (32, 64) lattice, first source, against the FP64 path
    i32 = lattices.index((32, 64))
    Sl, Ss = inputs[i32]
    c = b.cors[i32][0]
    o = torch.empty((N_CH, 32 ** 3, 16), dtype=torch.complex128, device=dev)
    c.run_each(Sl, Ss, [40], o)
    ref = bbc.Correlators(32, 64, 0, M_UD, M_S, channels=list(range(N_CH)), precision=bbc.BBC_FP64, device=dev)
    ro = torch.empty_like(o)
    ref.run_each(Sl, Ss, [40], ro)
    torch.cuda.synchronize(dev)
    err = channel_errors(torch, o, ro)
    ref.close()
    units = b.sites_channels()
    slices = sum(4 * T for _, T in lattices)
    b.close()
    from paper_1510_00903_gb300 import shard
    return {"value": shard.job_throughput(units, world, ms), "ms_per_step": round(ms, 2), "slices_per_step": slices,
            "workload": "8 lattices, L 16/24/32, T 32/48/64, 4 sources, mixed, complex64, one CUDA graph per step",
            "err_vs_fp64": err}


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    main()
