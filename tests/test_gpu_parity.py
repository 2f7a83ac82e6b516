"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerances: FP64 path 1e-12 of the per-slice, per-channel maximum |C|
(max over r and spin), the bound the paper's FP64 agreement suggests;
mixed path (FP32 blocks, FFTs and pair products, FP64 Wick-sign sums)
MIXED_TOL of the same scale, from the FP32 unit roundoff 6e-8 times the
growth of the sums (K <= 144 products, three FFT passes of 16-32 points, a
signed sum of up to 72 diagrams).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
import oracle.oracle as orc

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1510_00903_gb300 import bbc  # noqa: E402

FP64_TOL = 1e-12
MIXED_TOL = 2e-5
# bfloat16 trial (Fourier-space blocks rounded to 8-bit mantissas before the
# FP32 products): unit roundoff 2^-9 = 2e-3 per factor, so about 4e-3 per
# product before the sums; the bound leaves a factor ~5 for the growth of the
# signed sums over diagrams
BF16_TOL = 2e-2
# TF32 trial (tensor-core operands rounded once to TF32): unit roundoff 2^-11
# per operand, the same allowance for the sums as bfloat16
TF32_TOL = 5e-3


def gpu_run(L, T, t0, channels, S_l, S_s, times, precision=bbc.BBC_FP64, slices=1, normalised=False,
            on_device=True, dtype=torch.complex128):
    dev = torch.device("cuda")
    cor = bbc.Correlators(L, T, t0, 0.3, 0.4, channels=channels, precision=precision, slices=slices)
    times = list(times)
    # S_l, S_s hold every slice 0..T-1; pass the requested ones in order
    Sl = torch.from_numpy(np.ascontiguousarray(S_l[times])).to(dtype)
    Ss = torch.from_numpy(np.ascontiguousarray(S_s[times])).to(dtype)
    if on_device:
        Sl, Ss = Sl.to(dev), Ss.to(dev)
    else:
        Sl, Ss = Sl.pin_memory(), Ss.pin_memory()
    out = cor.run(Sl, Ss, times, normalised=normalised)
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    cor.close()
    return res


def rel_err(a, b):
    """max |a - b| / max |b| per channel; a, b: [n_ch, V or n_r, 16]."""
    scale = np.abs(b).reshape(b.shape[0], -1).max(axis=1)
    err = np.abs(a - b).reshape(b.shape[0], -1).max(axis=1)
    return err / np.where(scale > 0, scale, 1.0), scale


def oracle_slice(L, F, t, channels, r=None):
    return orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], channels, r)


# --------------------------------------------------------------------- config 1
def test_pLambda_L4_T4_full_grid_fp64():
    """p Lambda <- p Lambda, L=4, T=4, one wall source at t0=0, all r and t."""
    L, T = 4, 4
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=0)
    got = gpu_run(L, T, 0, [1], F["u"], F["s"], range(T))
    for t in range(T):
        e, _ = rel_err(got[t], oracle_slice(L, F, t, [1]))
        assert e.max() < FP64_TOL, (t, e)


def test_all_channels_L4_fp64_and_mixed():
    """All 52 channels, the 4 omitted ones and the 8 other charge states (all
    64 ids in one context), full grid of one slice."""
    L, T = 4, 4
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=1)
    ch = list(range(64))
    live = list(range(52)) + list(range(56, 64))
    want = oracle_slice(L, F, 3, ch)
    got = gpu_run(L, T, 0, ch, F["u"], F["s"], [3])[0]
    e, scale = rel_err(got[live], want[live])
    assert e.max() < FP64_TOL, e
    # omitted channels vanish (isospin limit) relative to the others
    assert np.abs(got[52:56]).max() < FP64_TOL * scale.max()
    gm = gpu_run(L, T, 0, ch, F["u"], F["s"], [3], precision=bbc.BBC_MIXED_FP32)[0]
    em, _ = rel_err(gm[live], want[live])
    assert em.max() < MIXED_TOL, em


@pytest.mark.parametrize("L", [4, 8])
def test_all_channels_bf16_trial(L):
    """The bfloat16 trial precision on one slice: all 52 channels at L = 4,
    twelve at L = 8 (oracle time)."""
    T = 4
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=11)
    ch = list(range(52)) if L == 4 else [0, 1, 5, 10, 14, 16, 27, 33, 41, 44, 48, 51]
    want = oracle_slice(L, F, 2, ch)
    got = gpu_run(L, T, 0, ch, F["u"], F["s"], [2], precision=bbc.BBC_MIXED_BF16)[0]
    e, _ = rel_err(got, want)
    print(f"bf16 L={L}: max {e.max():.3e} median {np.median(e):.3e}")
    assert e.max() < BF16_TOL, e
    assert np.median(e) > 1e-5  # the rounding is really applied


@pytest.mark.parametrize("L", [4, 8])
def test_all_channels_tf32_trial(L):
    """The TF32 trial precision (tensor-core products of single TF32 words)."""
    T = 4
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=12)
    ch = list(range(52)) if L == 4 else [0, 1, 5, 10, 14, 16, 27, 33, 41, 44, 48, 51]
    want = oracle_slice(L, F, 2, ch)
    got = gpu_run(L, T, 0, ch, F["u"], F["s"], [2], precision=bbc.BBC_MIXED_TF32)[0]
    e, _ = rel_err(got, want)
    print(f"tf32 L={L}: max {e.max():.3e} median {np.median(e):.3e}")
    assert e.max() < TF32_TOL, e
    assert np.median(e) > 1e-6  # the rounding is really applied


def test_L2_and_L8_slices_fp64():
    for L, chans in ((2, list(range(52))), (8, [0, 10, 27, 41, 51])):
        F = synth.flavour_set(L, 2, 0, 0.3, 0.4, seed=2)
        want = oracle_slice(L, F, 1, chans)
        got = gpu_run(L, 2, 0, chans, F["u"], F["s"], [1])[0]
        e, _ = rel_err(got, want)
        assert e.max() < FP64_TOL, (L, e)


def test_normalisation_and_host_input_and_c64():
    """Normalised output = raw x exp((m_B1+m_B2) d); host (pinned) input and
    complex64 input give the same result as device complex128 input of the
    same values."""
    L, T, t0 = 4, 8, 2
    F = synth.flavour_set(L, T, t0, 0.3, 0.4, seed=3)
    ch = [0, 1, 44, 51]
    times = [1, 5]
    raw = gpu_run(L, T, t0, ch, F["u"], F["s"], times)
    nrm = gpu_run(L, T, t0, ch, F["u"], F["s"], times, normalised=True, on_device=False)
    for i, t in enumerate(times):
        d = (t - t0) % T
        want = orc.normalise(oracle_slice(L, F, t, ch), ch, d, 0.3, 0.4)
        e, _ = rel_err(nrm[i], want)
        assert e.max() < FP64_TOL
        assert rel_err(raw[i], oracle_slice(L, F, t, ch))[0].max() < FP64_TOL
    F32 = {k: v.astype(np.complex64).astype(np.complex128) for k, v in F.items()}
    got = gpu_run(L, T, t0, ch, F32["u"], F32["s"], times, dtype=torch.complex64)
    for i, t in enumerate(times):
        assert rel_err(got[i], oracle_slice(L, F32, t, ch))[0].max() < FP64_TOL


def test_multi_slot_batch_equals_single():
    L, T = 4, 6
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=4)
    ch = [2, 13, 45]
    a = gpu_run(L, T, 0, ch, F["u"], F["s"], range(T), slices=1)
    b = gpu_run(L, T, 0, ch, F["u"], F["s"], range(T), slices=4)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()


# ---------------------------------------------------- closed form, any size
@pytest.mark.parametrize("L", [8, 16, 24, 32, 48])
def test_plane_wave_closed_form_all_channels(L):
    """Colour-diagonal plane waves: C(r) = V delta(P1+P2) e^{i P1.r} K, with K
    the single-site value from the oracle (property of Sec. 3 Eq.
    LN.pLLp.FFT holding at any L); only 5-light + 1-strange channels carry
    total momentum zero for the momenta chosen."""
    rng = np.random.default_rng(L)
    n_l = np.array([1, 2, 3])
    n_s = (-5 * n_l) % L
    P = {f: rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4)) for f in "ls"}
    Sl = synth.plane_wave(L, P["l"], n_l)[None]
    Ss = synth.plane_wave(L, P["s"], n_s)[None]  # one slice, t = 0
    ch = list(range(52))
    got = gpu_run(L, 1, 0, ch, Sl, Ss, [0])[0]
    S1 = {f: np.kron(P[f], np.eye(3))[None] for f in "ls"}
    K = orc.correlator(1, S1["l"], S1["l"], S1["s"], ch)[:, 0]  # [ch, 16]
    V = L ** 3
    r = np.arange(V)
    x, y, z = r % L, (r // L) % L, r // (L * L)
    content = {"p": "lll", "n": "lll", "Sigma+": "lsl", "Sigma-": "lsl", "Sigma0": "lsl",
               "Lambda": "lsl", "Xi0": "lss", "Xi-": "lss"}
    scale = V * np.abs(K).max()
    for c in ch:
        b = orc.channel_baryons(c)
        q1 = content[b[0]]
        tot = sum(content[x_].count("s") for x_ in b[:2])
        if tot == 1:
            P1 = q1.count("l") * n_l + q1.count("s") * n_s
            ph = np.exp(2j * np.pi * (P1[0] * x + P1[1] * y + P1[2] * z) / L)
            want = V * ph[:, None] * K[c][None, :]
            assert np.abs(got[c] - want).max() < FP64_TOL * max(np.abs(want).max(), 1e-300), c
        else:
            assert np.abs(got[c]).max() < FP64_TOL * scale, c


# ------------------------------------------------ sampled points, radix 3
def test_L24_radix3_sampled_fp64():
    """L = 24 (radix-3 transforms) against the oracle on sampled r (the
    full-size lattices are checked against stored oracle values in
    test_gpu_golden_parity.py)."""
    L, T, t = 24, 4, 2
    chans = [0, 10, 51]
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=8, times=[t])
    r_list = [0, 1, 24 * 24 * 5 + 24 * 13 + 7]
    want = orc.correlator(L, F["u"][0], F["d"][0], F["s"][0], chans, r_list)
    cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=chans, precision=bbc.BBC_FP64)
    dev = torch.device("cuda")
    out = cor.run(torch.from_numpy(F["u"]).to(dev), torch.from_numpy(F["s"]).to(dev), [t], normalised=False)
    torch.cuda.synchronize()
    g = out[0].cpu().numpy()
    cor.close()
    e, _ = rel_err(g[:, r_list], want)  # scale: the oracle's maximum per channel
    assert e.max() < FP64_TOL, e
