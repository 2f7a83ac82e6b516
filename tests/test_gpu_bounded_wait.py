"""The queue-driven forward FFT of the mixed precisions (GPU).

* Parity: its output, through the whole mixed path, against the FP64 path
  (field-major FFT passes, pinned to the oracle elsewhere) at every L it
  serves, with ragged row tiles and two slots per launch.
* Bounded waits: the self-test gives the z-line units a dependency count no
  plane unit reaches; each wait runs out after its poll limit, the kernel
  records the timeout in the context's status word and stops, the host reads
  BBC_ETIMEOUT, and the context stays usable.  Nothing faults, traps or spins
  without a limit.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1510_00903_gb300 import bbc  # noqa: E402

CHANS = [0, 10, 51]  # 4912 block rows: ragged tiles of 32, 16 and 8 columns
MIXED_TOL = 2e-5


def _inputs(L, T, seed, dev):
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=seed)
    return torch.from_numpy(F["u"]).to(dev), torch.from_numpy(F["s"]).to(dev)


@pytest.mark.parametrize("L", [2, 4, 8, 16, 24, 32])
def test_queue_fft_mixed_path_matches_fp64_path(L):
    dev = torch.device("cuda", torch.cuda.current_device())
    T = 4
    Sl, Ss = _inputs(L, T, 90 + L, dev)
    times = [1, 2]
    ref = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=CHANS, precision=bbc.BBC_FP64, device=dev)
    want = ref.run(Sl, Ss, times).cpu().numpy()
    ref.close()
    mix = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=CHANS, precision=bbc.BBC_MIXED_FP32, slices=2, device=dev)
    assert bbc.bbc_launch_counts(mix.ctx)["build"] == 2  # block build + one queue-driven FFT launch
    got = mix.run(Sl, Ss, times).cpu().numpy()
    mix.status()
    mix.close()
    # per (slice, channel): relative to the largest correlator value
    scale = np.abs(want).max(axis=(2, 3), keepdims=True)
    err = (np.abs(got - want) / scale).max()
    assert err < MIXED_TOL, err


def test_bounded_wait_runs_out_and_the_context_recovers():
    dev = torch.device("cuda", torch.cuda.current_device())
    L, T = 8, 4
    Sl, Ss = _inputs(L, T, 77, dev)
    cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=CHANS, precision=bbc.BBC_MIXED_FP32, device=dev)
    before = cor.run(Sl, Ss, [1]).clone()
    cor.status()  # no wait gave up
    t0 = time.perf_counter()
    st = bbc.bbc_check_bounded_wait(cor.ctx, 20000)  # about 10 ms of polls per wait
    elapsed = time.perf_counter() - t0
    assert st == bbc.BBC_ETIMEOUT, (st, bbc.lib().bbc_last_error(cor.ctx))
    assert "bounded wait" in bbc.lib().bbc_last_error(cor.ctx).decode()
    assert elapsed < 30.0
    # the self-test left slot 0 unbuilt: contracting it now is out of order
    out = torch.empty((len(CHANS), L ** 3, 16), dtype=torch.complex128, device=dev)
    with pytest.raises(bbc.BBCError) as e:
        cor.contract(0, out)
    assert e.value.status == bbc.BBC_ESTATE
    cor.status()  # the record was read and cleared
    after = cor.run(Sl, Ss, [1])
    cor.status()
    torch.cuda.synchronize(dev)
    scale = before.abs().amax(dim=(-2, -1), keepdim=True)
    assert ((after - before).abs() / scale).max().item() < 1e-5  # FP32 atomics order only
    cor.close()


def test_bounded_wait_self_test_needs_the_queue_driven_fft():
    dev = torch.device("cuda", torch.cuda.current_device())
    cor = bbc.Correlators(8, 4, 0, 0.3, 0.4, channels=[0], precision=bbc.BBC_FP64, device=dev)
    assert bbc.bbc_check_bounded_wait(cor.ctx, 1000) == bbc.BBC_ESTATE
    cor.close()
