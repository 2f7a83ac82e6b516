"""GPU parity at the full-size lattices against stored oracle values.

The expected values are the CPU FP64 oracle's correlators at sampled r,
written by ``golden/make_oracle_goldens.py`` (which imports only ``synth``
and ``oracle``).  The inputs are rebuilt here with the same generator tags
and checked against the stored checksum first, so a failure names either the
generator or the kernels.  Every comparison is element by element at the
stored (channel, r, spin) points, scaled per channel and slice by the
oracle's own maximum |C| over those points -- never by the GPU output.

Tolerances (relative to that scale): FP64 and double-float 1e-12; the mixed
FP32 path 2e-5 (FP32 unit roundoff 6e-8 grown by K <= 144 products, three FFT
passes and signed sums over up to 72 diagrams); the bfloat16 trial 2e-2;
the TF32 trial 5e-3 (unit roundoff 2^-11 = 4.9e-4 per operand, so about
1e-3 per product, with the same allowance for the sums as bfloat16).
The launch configurations are those the benchmark times (autotuned shapes,
all slices of a source in one call, the batch as one captured graph, the
48^3 lattice streamed from pinned host memory).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
import oracle.oracle as orc

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1510_00903_gb300 import bbc  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
FP64_TOL, MIXED_TOL, BF16_TOL, TF32_TOL = 1e-12, 2e-5, 2e-2, 5e-3


def golden(name):
    path = os.path.join(HERE, "golden", f"oracle_{name}.npz")
    if not os.path.exists(path):
        pytest.fail(f"missing {path}: run tests/golden/make_oracle_goldens.py {name}")
    g = np.load(path)
    return {k: g[k] for k in g.files}


def slice_inputs(g, t, all_slices=False):
    """Propagators of the golden case (light, strange), [n_t, V, 12, 12]
    complex128 holding the stored precision's values; all T slices or slice t."""
    L, T, t0 = int(g["L"]), int(g["T"]), int(g["t0"])
    times = list(range(T)) if all_slices else [t]
    F = synth.flavour_set(L, T, t0, float(g["m_ud"]), float(g["m_s"]), seed=int(g["seed"]),
                          lattice=int(g["lattice"]), source=int(g["source"]), times=times)
    Sl, Ss = F["u"], F["s"]
    if str(g["storage"]) == "c64":
        Sl = Sl.astype(np.complex64).astype(np.complex128)
        Ss = Ss.astype(np.complex64).astype(np.complex128)
    return Sl, Ss


def check_inputs(g, i, Sl, Ss):
    chk = g["checksum"][i]
    got = [float(np.sum(np.abs(Sl) ** 2)), float(np.sum(np.abs(Ss) ** 2))]
    assert np.allclose(got, chk, rtol=1e-12, atol=0), ("generator changed", got, chk)


def errors(got, want):
    """Per channel: max over the stored points of |got - want| / max |want|."""
    scale = np.abs(want).reshape(want.shape[0], -1).max(axis=1)
    assert (scale > 0).all()
    return np.abs(got - want).reshape(want.shape[0], -1).max(axis=1) / scale


# ------------------------------------------------- 16^3 x 32, all 32 slices
@pytest.mark.parametrize("precision,tol", [(bbc.BBC_FP64, FP64_TOL), (bbc.BBC_DF64, FP64_TOL),
                                           (bbc.BBC_MIXED_FP32, MIXED_TOL)], ids=["fp64", "df64", "mixed"])
def test_L16_T32_all_channels_four_slices(precision, tol):
    """The 52-channel bench lattice: every slice of the source in one call with
    autotuned shapes; four slices checked at 64 r, raw and normalised."""
    g = golden("config2_L16_T32")
    L, T, t0 = int(g["L"]), int(g["T"]), int(g["t0"])
    dev = torch.device("cuda", torch.cuda.current_device())
    Sl, Ss = slice_inputs(g, None, all_slices=True)
    for i, t in enumerate(g["slices"]):
        check_inputs(g, i, Sl[t], Ss[t])
    Sl, Ss = torch.from_numpy(Sl).to(dev), torch.from_numpy(Ss).to(dev)
    chans = [int(c) for c in g["channels"]]
    cor = bbc.Correlators(L, T, t0, float(g["m_ud"]), float(g["m_s"]), channels=chans, precision=precision,
                          device=dev)
    cor.autotune(Sl[0], Ss[0], t=0, reps=1)
    raw = cor.run(Sl, Ss, range(T), normalised=False)
    nrm = cor.run(Sl, Ss, range(T), normalised=True)
    torch.cuda.synchronize()
    r = torch.from_numpy(g["r"].astype(np.int64)).to(dev)
    worst = 0.0
    for i, t in enumerate(g["slices"]):
        want = g["C"][i]
        e = errors(raw[int(t)][:, r].cpu().numpy(), want)
        assert e.max() < tol, (int(t), e)
        d = (int(t) - t0) % T
        en = errors(nrm[int(t)][:, r].cpu().numpy(), orc.normalise(want, chans, d, float(g["m_ud"]), float(g["m_s"])))
        assert en.max() < tol, (int(t), en)
        worst = max(worst, e.max(), en.max())
    print(f"L16 precision {precision}: max error {worst:.2e}")
    cor.close()


# ----------------------------------------------------------- 32^3 x 64, t = 32
@pytest.mark.parametrize("precision,tol", [(bbc.BBC_FP64, FP64_TOL), (bbc.BBC_DF64, FP64_TOL),
                                           (bbc.BBC_MIXED_FP32, MIXED_TOL), (bbc.BBC_MIXED_BF16, BF16_TOL),
                                           (bbc.BBC_MIXED_TF32, TF32_TOL)],
                         ids=["fp64", "df64", "mixed", "bf16", "tf32"])
def test_L32_T64_all_channels(precision, tol):
    g = golden("config3_L32_T64")
    L, T, t0 = int(g["L"]), int(g["T"]), int(g["t0"])
    t = int(g["slices"][0])
    dev = torch.device("cuda", torch.cuda.current_device())
    Sl, Ss = slice_inputs(g, t)
    check_inputs(g, 0, Sl[0], Ss[0])
    chans = [int(c) for c in g["channels"]]
    cor = bbc.Correlators(L, T, t0, float(g["m_ud"]), float(g["m_s"]), channels=chans, precision=precision,
                          device=dev)
    out = cor.run(torch.from_numpy(Sl).to(dev), torch.from_numpy(Ss).to(dev), [t], normalised=False)
    r = torch.from_numpy(g["r"].astype(np.int64)).to(dev)
    got = out[0][:, r].cpu().numpy()
    cor.close()
    e = errors(got, g["C"][0])
    print(f"L32 precision {precision}: max error {e.max():.2e}, median {np.median(e):.2e}")
    assert e.max() < tol, e
    if precision in (bbc.BBC_MIXED_BF16, bbc.BBC_MIXED_TF32):
        assert np.median(e) > 1e-6  # the rounding is applied


# ------------------------------------------- two items of the uneven batch
def test_batch_items_L24_L32_captured_graph():
    """Items of the uneven batch (complex64 propagators, mixed precision, wall
    sources at t0 = T/4 and T/2) through bbc_batch_run, captured as one CUDA
    graph and replayed twice; checked against the oracle at sampled r."""
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(dev)
    cases = [golden("config4_L24_T48"), golden("config4_L32_T64")]
    cors, keep, outs = [], [], []
    items = (bbc.bbc_batch_item * len(cases))()
    for k, g in enumerate(cases):
        L, T, t0, t = int(g["L"]), int(g["T"]), int(g["t0"]), int(g["slices"][0])
        Sl, Ss = slice_inputs(g, t)
        check_inputs(g, 0, Sl[0], Ss[0])
        c = bbc.Correlators(L, T, t0, float(g["m_ud"]), float(g["m_s"]), channels=[int(x) for x in g["channels"]],
                            precision=bbc.BBC_MIXED_FP32, device=dev, stream=stream)
        dl = torch.from_numpy(Sl[0]).to(torch.complex64).to(dev)
        ds = torch.from_numpy(Ss[0]).to(torch.complex64).to(dev)
        out = torch.zeros((len(g["channels"]), L ** 3, 16), dtype=torch.complex128, device=dev)
        items[k] = bbc.bbc_batch_item(c.ctx, t, dl.data_ptr(), ds.data_ptr(), bbc.BBC_C64, 1, out.data_ptr(), 0)
        cors.append(c)
        keep += [dl, ds]
        outs.append(out)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        bbc.bbc_batch_run(items, len(cases), stream.cuda_stream)  # eager run: kernel attributes
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        bbc.bbc_batch_run(items, len(cases), stream.cuda_stream)
    for o in outs:
        o.zero_()
    for rep in range(2):
        graph.replay()
        torch.cuda.synchronize()
        for g, o in zip(cases, outs):
            r = torch.from_numpy(g["r"].astype(np.int64)).to(dev)
            e = errors(o[:, r].cpu().numpy(), g["C"][0])
            assert e.max() < MIXED_TOL, (int(g["L"]), rep, e)
    for c in cors:
        c.close()


# ---------------------------------------------------- 48^3 x 96, streamed
def test_L48_streamed_mixed_fp64_df64():
    """The 48^3 lattice: complex64 propagators in pinned host memory copied per
    slice (run_streamed, mixed precision), and the FP64 and double-float paths
    on the same values, against the oracle at sampled r (three channels)."""
    g = golden("config5_L48_T96")
    L, T, t0 = int(g["L"]), int(g["T"]), int(g["t0"])
    t = int(g["slices"][0])
    dev = torch.device("cuda", torch.cuda.current_device())
    Sl, Ss = slice_inputs(g, t)
    check_inputs(g, 0, Sl[0], Ss[0])
    chans = [int(c) for c in g["channels"]]
    r = torch.from_numpy(g["r"].astype(np.int64)).to(dev)
    # host [T, V, 12, 12] views holding slice t (only slice t is read)
    hl = torch.zeros((t + 1, L ** 3, 12, 12), dtype=torch.complex64).pin_memory()
    hs = torch.zeros_like(hl).pin_memory()
    hl[t].copy_(torch.from_numpy(Sl[0]))
    hs[t].copy_(torch.from_numpy(Ss[0]))
    cor = bbc.Correlators(L, T, t0, float(g["m_ud"]), float(g["m_s"]), channels=chans,
                          precision=bbc.BBC_MIXED_FP32, device=dev, stream=torch.cuda.Stream(dev))
    out = torch.empty((len(chans), L ** 3, 16), dtype=torch.complex128, device=dev)
    cor.run_streamed(hl, hs, [t], out, normalised=False)
    torch.cuda.synchronize()
    em = errors(out[:, r].cpu().numpy(), g["C"][0])
    cor.close()
    assert em.max() < MIXED_TOL, em
    for prec in (bbc.BBC_FP64, bbc.BBC_DF64):  # FP64 and double-float: 48-point lines split over three threads
        ref = bbc.Correlators(L, T, t0, float(g["m_ud"]), float(g["m_s"]), channels=chans, precision=prec,
                              device=dev)
        o64 = ref.run(torch.from_numpy(Sl).to(dev), torch.from_numpy(Ss).to(dev), [t], normalised=False)
        torch.cuda.synchronize()
        e64 = errors(o64[0][:, r].cpu().numpy(), g["C"][0])
        ref.close()
        del o64
        assert e64.max() < FP64_TOL, (prec, e64)
