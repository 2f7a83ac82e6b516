"""CUDA-graph capture of the whole slice loop, and several lattices with
uneven L and T run as one graph (GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
import oracle.oracle as orc

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1510_00903_gb300 import bbc  # noqa: E402


@pytest.mark.parametrize("precision", [bbc.BBC_FP64, bbc.BBC_MIXED_FP32])
def test_graph_replay_equals_eager(precision):
    L, T = 8, 4
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=31)
    Sl, Ss = torch.from_numpy(F["u"]).to(dev), torch.from_numpy(F["s"]).to(dev)
    cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=[0, 10, 51], precision=precision, device=dev,
                          stream=torch.cuda.Stream(dev))
    eager = cor.run(Sl, Ss, range(T)).clone()
    torch.cuda.synchronize(dev)
    out = torch.zeros_like(eager)
    g = cor.capture(Sl, Ss, range(T), out)
    out.zero_()
    g.replay()
    torch.cuda.synchronize(dev)
    if precision == bbc.BBC_FP64:
        assert torch.equal(out, eager)  # same kernels, same order, no atomics
    else:
        # the FP32 products are added into shared memory with atomics, whose
        # order varies from run to run at the FP32 rounding level
        scale = eager.abs().amax(dim=(-2, -1), keepdim=True)
        assert ((out - eager).abs() / scale).max().item() < 1e-5
    cor.close()


def test_lattice_batch_uneven_lattices_one_graph():
    """Two lattices of different L and T and two sources each in one graph;
    the last slice of each lattice matches the oracle (mixed tolerance)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    lat = [(4, 4), (8, 6)]
    inputs, Fs = [], []
    for i, (L, T) in enumerate(lat):
        F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=40 + i)
        Fs.append(F)
        inputs.append((torch.from_numpy(F["u"]).to(torch.complex64).to(dev),
                       torch.from_numpy(F["s"]).to(torch.complex64).to(dev)))
    chans = [1, 41]
    b = bbc.LatticeBatch(lat, inputs, n_sources=2, channels=chans, precision=bbc.BBC_MIXED_FP32, device=dev)
    g = b.capture()
    for o in b.outputs:
        o.zero_()
    g.replay()
    torch.cuda.synchronize(dev)
    for (L, T), F, o in zip(lat, Fs, b.outputs):
        t, t0 = T - 1, T // 2  # last slice of the second source
        F32 = {k: v.astype(np.complex64).astype(np.complex128) for k, v in F.items()}
        want = orc.normalise(orc.correlator(L, F32["u"][t], F32["d"][t], F32["s"][t], chans), chans,
                             (t - t0) % T, 0.3, 0.4)
        got = o.cpu().numpy()
        scale = np.abs(want).reshape(len(chans), -1).max(axis=1)
        err = np.abs(got - want).reshape(len(chans), -1).max(axis=1) / scale
        assert err.max() < 2e-5, (L, err)
    assert b.sites_channels() == 2 * (4 * 64 + 6 * 512) * 2
    b.close()


def test_run_streamed_overlapped_copies():
    """Pinned host propagators streamed slice by slice (copy of slice t+1
    overlapping slice t): every slice equals the oracle."""
    L, T = 8, 5
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=61)
    chans = [1, 41]
    Sl = torch.from_numpy(F["u"]).to(torch.complex64).pin_memory()
    Ss = torch.from_numpy(F["s"]).to(torch.complex64).pin_memory()
    cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=chans, precision=bbc.BBC_MIXED_FP32, device=dev,
                          stream=torch.cuda.Stream(dev))
    out = torch.empty((len(chans), L ** 3, 16), dtype=torch.complex128, device=dev)
    res = torch.empty((T,) + tuple(out.shape), dtype=out.dtype, device=dev)
    cor.run_streamed(Sl, Ss, range(T), out, on_slice=lambda t, o: res[t].copy_(o))
    torch.cuda.synchronize(dev)
    got = res.cpu().numpy()
    for t in range(T):
        F32 = {k: v[t].astype(np.complex64).astype(np.complex128) for k, v in F.items()}
        want = orc.normalise(orc.correlator(L, F32["u"], F32["d"], F32["s"], chans), chans, t, 0.3, 0.4)
        scale = np.abs(want).reshape(len(chans), -1).max(axis=1)
        err = np.abs(got[t] - want).reshape(len(chans), -1).max(axis=1) / scale
        assert err.max() < 2e-5, (t, err)
    cor.close()


def test_numeric_checks():
    """BBC_CHECK_INPUT flags a NaN propagator entry, BBC_CHECK_OUTPUT the NaN
    correlators it produces; finite data passes both."""
    L, T = 4, 2
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=71)
    Sl, Ss = torch.from_numpy(F["u"]).to(dev), torch.from_numpy(F["s"]).to(dev)
    cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=[0], device=dev)
    bbc.bbc_set_checks(cor.ctx, bbc.BBC_CHECK_INPUT | bbc.BBC_CHECK_OUTPUT)
    cor.run(Sl, Ss, range(T))  # finite: no error
    bad = Sl.clone()
    bad[1, 5, 3, 7] = complex(float("nan"), 0.0)
    with pytest.raises(bbc.BBCError) as e:
        cor.run(bad[1:2], Ss[1:2], [1])  # propagators of the listed slices, in order
    assert e.value.status == bbc.BBC_ENUMERIC and "light" in str(e.value)
    bbc.bbc_set_checks(cor.ctx, bbc.BBC_CHECK_OUTPUT)
    with pytest.raises(bbc.BBCError) as e:
        cor.run(bad[1:2], Ss[1:2], [1])
    assert e.value.status == bbc.BBC_ENUMERIC and "correlators" in str(e.value)
    torch.cuda.synchronize(dev)
    cor.close()


def test_run_to_host_end_to_end():
    """Pinned host in, pinned host out, copies overlapped with the compute:
    every slice equals the oracle."""
    L, T = 4, 5
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, 1, 0.3, 0.4, seed=63)
    chans = [0, 51]
    Sl = torch.from_numpy(F["u"]).pin_memory()
    Ss = torch.from_numpy(F["s"]).pin_memory()
    cor = bbc.Correlators(L, T, 1, 0.3, 0.4, channels=chans, device=dev, stream=torch.cuda.Stream(dev))
    out = torch.empty((T, len(chans), L ** 3, 16), dtype=torch.complex128).pin_memory()
    cor.run_to_host(Sl, Ss, range(T), out)
    torch.cuda.synchronize(dev)
    for t in range(T):
        want = orc.normalise(orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], chans), chans, (t - 1) % T, 0.3, 0.4)
        scale = np.abs(want).reshape(len(chans), -1).max(axis=1)
        err = np.abs(out[t].numpy() - want).reshape(len(chans), -1).max(axis=1) / scale
        assert err.max() < 1e-12, (t, err)
    cor.close()


def test_batch_failure_names_the_item_and_resumes():
    """Failure and resume of a batch without any device fault: item 2 asks for
    a time slice outside the lattice, so bbc_batch_run returns EINVAL naming
    item 2 after items 0 and 1 ran, and item 2 writes nothing.  Work items are
    independent, so running the batch again from item 2 (slice fixed)
    completes it; every output equals the eager run of the same context."""
    L, T = 4, 4
    chans = [1, 41]
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=44)
    Sl, Ss = torch.from_numpy(F["u"]).to(dev), torch.from_numpy(F["s"]).to(dev)
    cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=chans, precision=bbc.BBC_FP64, device=dev)
    want = cor.run(Sl, Ss, range(T)).cpu().numpy()
    outs = [torch.zeros((len(chans), L ** 3, 16), dtype=torch.complex128, device=dev) for _ in range(T)]
    items = (bbc.bbc_batch_item * T)()
    for t in range(T):
        items[t] = bbc.bbc_batch_item(cor.ctx, t, Sl[t].data_ptr(), Ss[t].data_ptr(), bbc.BBC_C128, 1,
                                      outs[t].data_ptr(), 1)
    items[2].t = T  # outside 0 <= t < T
    stream = torch.cuda.current_stream(dev)
    with pytest.raises(bbc.BBCError) as e:
        bbc.bbc_batch_run(items, T, stream.cuda_stream)
    assert e.value.status == bbc.BBC_EINVAL and "batch item 2" in str(e.value)
    torch.cuda.synchronize(dev)

    def close(t):
        got = outs[t].cpu().numpy()
        return np.abs(got - want[t]).max() <= 1e-14 * np.abs(want[t]).max()

    assert close(0) and close(1)
    assert outs[2].abs().max().item() == 0 and outs[3].abs().max().item() == 0
    items[2].t = 2
    rest = (bbc.bbc_batch_item * (T - 2))(*[items[i] for i in range(2, T)])
    bbc.bbc_batch_run(rest, T - 2, stream.cuda_stream)
    torch.cuda.synchronize(dev)
    assert all(close(t) for t in range(T))
    cor.close()
