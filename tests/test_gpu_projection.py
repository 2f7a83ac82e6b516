"""Parity of bbc_project (spin states |J M> and the cubic-group A1 average of
Sec. 2) with the projection oracle (GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
import oracle.oracle as orc
from oracle import projection as pj

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1510_00903_gb300 import bbc  # noqa: E402

TOL = 1e-13  # FP64 sums of 24 terms and one 1/sqrt2 scaling: a few ulps


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("L,n_fields", [(2, 1), (4, 3), (8, 2), (16, 2), (24, 1), (32, 1)])
def test_project_random_fields(L, n_fields):
    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(L)
    C = rng.normal(size=(n_fields, L ** 3, 16)) + 1j * rng.normal(size=(n_fields, L ** 3, 16))
    cor = bbc.Correlators(L, 4, 0, 0.3, 0.4, channels=[0], device=dev)
    R, Ra1 = cor.project(torch.from_numpy(C).to(dev))
    torch.cuda.synchronize(dev)
    want_R = pj.project_spin(C)
    want_A = pj.project_a1(want_R, L)
    assert _rel(R.cpu().numpy(), want_R) < TOL
    assert _rel(Ra1.cpu().numpy(), want_A) < TOL
    # spin states only
    R2, none = cor.project(torch.from_numpy(C).to(dev), a1=False)
    torch.cuda.synchronize(dev)
    assert none is None and _rel(R2.cpu().numpy(), want_R) < TOL
    cor.close()


def test_project_correlators_end_to_end():
    """Correlators of identical-source channels through the whole GPU path,
    then projected: parity with oracle(correlator) -> oracle(projection), and
    the J = 1 states vanish (the Pauli zero of two equal source baryons)."""
    L, T, t = 4, 4, 2
    dev = torch.device("cuda", torch.cuda.current_device())
    F = synth.flavour_set(L, T, 0, 0.3, 0.4, seed=23)
    chans = [10, 1, 37]  # Lambda Lambda <- Lambda Lambda, p Lambda <- p Lambda, Sigma0 Sigma0 <- Sigma0 Sigma0
    cor = bbc.Correlators(L, T, 0, 0.3, 0.4, channels=chans, device=dev)
    C = cor.run(torch.from_numpy(F["u"][t:t + 1]).to(dev), torch.from_numpy(F["s"][t:t + 1]).to(dev), [t])[0]
    R, Ra1 = cor.project(C)
    torch.cuda.synchronize(dev)
    want_C = orc.normalise(orc.correlator(L, F["u"][t], F["d"][t], F["s"][t], chans), chans, t, 0.3, 0.4)
    want_R = pj.project_spin(want_C)
    want_A = pj.project_a1(want_R, L)
    got_R, got_A = R.cpu().numpy(), Ra1.cpu().numpy()
    for i in range(len(chans)):
        assert _rel(got_R[i], want_R[i]) < 1e-12
        assert _rel(got_A[i], want_A[i]) < 1e-12
    for i in (0, 2):
        assert np.abs(got_R[i, :, 4:]).max() <= 1e-12 * np.abs(got_R[i]).max()
    cor.close()
