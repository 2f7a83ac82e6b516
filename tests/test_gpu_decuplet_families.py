"""GPU parity of the other decuplet channels of the Sec. 4 footnote (Gamma1 =
C gamma_l, Gamma2 = 1): Delta++ Delta++, Sigma*+ Sigma*+, Xi*0 Xi*0 (81 vector
combinations each, ids 154..396) and p Delta++ (ids 397..405), through the C ABI
against the oracle.  They bring the (l, l) and (l, s) vector diquarks, the
(l l l), (l l s), (l s l), (l s s) and (s s l) vector families and the two-term
Sigma*+ / Xi*0 operators into the block build.

Tolerances as for the octet channels: FP64 and double-float 1e-12 of the
per-channel maximum; mixed (FP32 products, double-float Wick sums) 2e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
import oracle.oracle as orc

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1510_00903_gb300 import bbc  # noqa: E402

FP64_TOL, MIXED_TOL = 1e-12, 2e-5
FAMILIES = {"Delta++ and p Delta++": bbc.DELTA_DELTA + bbc.P_DELTA, "Sigma*+ pairs": bbc.SIGMA_STAR_PAIRS,
            "Xi*0 pairs": bbc.XI_STAR_PAIRS}


def _err(got, want):
    scale = np.abs(want).reshape(want.shape[0], -1).max(axis=1)
    return np.abs(got - want).reshape(want.shape[0], -1).max(axis=1) / np.where(scale > 0, scale, 1.0)


def _run(L, T, t0, chans, F, t, precision=bbc.BBC_FP64, components=bbc.BBC_UPPER, normalised=False, k=None):
    """Slice t of the lattice; its propagators are F[...][k] (k = t unless given)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    cor = bbc.Correlators(L, T, t0, 0.3, 0.4, channels=chans, precision=precision, device=dev,
                          components=components)
    k = t if k is None else k
    Sl = torch.from_numpy(np.ascontiguousarray(F["u"][k:k + 1])).to(dev)
    Ss = torch.from_numpy(np.ascontiguousarray(F["s"][k:k + 1])).to(dev)
    out = cor.run(Sl, Ss, [t], normalised=normalised)[0].cpu().numpy()
    cor.close()
    return out


@pytest.fixture(scope="module")
def families_L4():
    L, T, t = 4, 4, 2
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=95)
    want = {name: orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], ids) for name, ids in FAMILIES.items()}
    return L, T, t, F, want


@pytest.mark.parametrize("family", list(FAMILIES))
@pytest.mark.parametrize("precision,tol", [(bbc.BBC_FP64, FP64_TOL), (bbc.BBC_DF64, FP64_TOL),
                                           (bbc.BBC_MIXED_FP32, MIXED_TOL)])
def test_family_all_ids_L4(families_L4, family, precision, tol):
    """Every id of a family in one context, every r of one slice."""
    L, T, t, F, want = families_L4
    ids = FAMILIES[family]
    got = _run(L, T, 0, ids, F, t, precision)
    e = _err(got, want[family])
    assert e.max() < tol, (e.max(), ids[int(e.argmax())])
    assert np.abs(want[family]).reshape(len(ids), -1).max(axis=1).min() > 0


def test_every_family_in_one_context():
    """Octet, Omega and the new decuplet families side by side in one block
    build (sixteen row groups, eleven diquarks per site), normalised."""
    L, T, t0, t = 4, 6, 1, 4
    F = synth.flavour_set(L, T, t0, 0.3, 0.4, seed=96)
    chans = [0, 10, 51, 64, 150, 154, 200, 240, 300, 320, 396, 400]
    raw = orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], chans)
    want = orc.normalise(raw, chans, t - t0, 0.3, 0.4)
    for precision, tol in ((bbc.BBC_FP64, FP64_TOL), (bbc.BBC_MIXED_FP32, MIXED_TOL)):
        got = _run(L, T, t0, chans, F, t, precision, normalised=True)
        e = _err(got, want)
        assert e.max() < tol, (precision, e)


@pytest.mark.parametrize("precision,tol", [(bbc.BBC_FP64, FP64_TOL), (bbc.BBC_MIXED_FP32, MIXED_TOL)])
def test_lower_components(precision, tol):
    """Lower Dirac components (Sec. 5) of the new families."""
    L, T, t0, t = 4, 6, 1, 4
    F = synth.flavour_set(L, T, t0, 0.3, 0.4, seed=97)
    chans = [154, 190, 235, 281, 316, 377, 401]
    got = _run(L, T, t0, chans, F, t, precision, components=bbc.BBC_LOWER)
    want = orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], chans, lower=True)
    e = _err(got, want)
    assert e.max() < tol, e


def test_L16_sampled():
    """L = 16 (the bench lattice), sampled r, the oracle's scale."""
    L, T, t = 16, 8, 3
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=98, times=[t])
    chans = [154, 235, 262, 316, 343, 405]
    rs = [0, 1, 17, 273, 2080, 4095]
    want = orc.correlator(L, F["u"][0], F["d"][0], F["s"][0], chans, rs)
    scale = np.abs(want).reshape(len(chans), -1).max(axis=1)
    for precision, tol in ((bbc.BBC_FP64, FP64_TOL), (bbc.BBC_DF64, FP64_TOL)):
        got = _run(L, T, 0, chans, F, t, precision, k=0)
        err = np.abs(got[:, rs] - want).reshape(len(chans), -1).max(axis=1) / scale
        assert err.max() < tol, (precision, err)
