"""Pins of the projection oracle (Sec. 2: source spin states |J M> and the
cubic-group operator P of the 3S1 / 3D1 split) against facts fixed
independently of it: angular-momentum algebra built from the Pauli
matrices, closed forms on the periodic lattice, and the Pauli principle for
identical source baryons."""
import math

import numpy as np
import pytest

import oracle.oracle as orc
from oracle import projection as pj
import synth


# ------------------------------------------------------------- spin states
def _spin_ops():
    """S_z, S_- and S^2 of two spin-1/2 particles acting on v[a', b']
    (index 0 = up), written from the Pauli matrices."""
    sz = np.diag([0.5, -0.5])
    sm = np.array([[0.0, 0.0], [1.0, 0.0]])          # lowers up -> down
    sp = sm.T
    sx, sy = 0.5 * (sp + sm), -0.5j * (sp - sm)
    def tot(op):
        return lambda v: op @ v + v @ op.T
    Sx, Sy, Sz, Sm = tot(sx), tot(sy), tot(sz), tot(sm)
    def S2(v):
        return Sx(Sx(v)) + Sy(Sy(v)) + Sz(Sz(v))
    return Sz, Sm, S2


def test_spin_states_are_angular_momentum_eigenstates():
    P = pj.spin_projector()
    Sz, Sm, S2 = _spin_ops()
    for jm, (J, M) in enumerate(pj.SPIN_STATES):
        v = P[jm]
        assert np.allclose(S2(v), J * (J + 1) * v, atol=1e-14)
        assert np.allclose(Sz(v), M * v, atol=1e-14)
        assert abs(np.vdot(v, v) - 1) < 1e-14
    # Condon-Shortley phases: S_- |1,1> = sqrt2 |1,0>, S_- |1,0> = sqrt2 |1,-1>
    assert np.allclose(Sm(P[1]), math.sqrt(2) * P[2], atol=1e-14)
    assert np.allclose(Sm(P[2]), math.sqrt(2) * P[3], atol=1e-14)
    assert np.allclose(Sm(P[0]), 0, atol=1e-14)
    G = np.einsum("ipq,jpq->ij", P, P)
    assert np.allclose(G, np.eye(4), atol=1e-14)


def test_project_spin_index_convention():
    """A product correlator u_{ab} w_{a'b'}, written with explicit index
    loops in the documented order, projects to u_{ab} <P_jm, w>."""
    rng = np.random.default_rng(5)
    P = pj.spin_projector()
    for k in range(4):
        u = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
        C = np.zeros((3, 16), complex)
        for a in range(2):
            for b in range(2):
                for ap in range(2):
                    for bp in range(2):
                        C[:, a + 2 * (b + 2 * (ap + 2 * bp))] = u[a, b] * P[k, ap, bp] * np.array([1, 2j, -3])
        R = pj.project_spin(C)
        for jm in range(4):
            for a in range(2):
                for b in range(2):
                    want = u[a, b] * (1.0 if jm == k else 0.0) * np.array([1, 2j, -3])
                    assert np.allclose(R[:, a + 2 * b + 4 * jm], want, atol=1e-14)


def test_identical_source_is_spin_singlet():
    """Two identical baryons created at one wall source obey the Pauli
    principle (Sec. 4, the identical-source zeros): the source pair is
    antisymmetric in (a', b'), so every J = 1 projection vanishes and the
    J = 0 one does not."""
    L = 2
    F = synth.flavour_set(L, 1, 0, 0.3, 0.4, seed=17)
    names = [orc.channel_name(c) for c in range(orc.n_channels())]
    same = [c for c in range(52) if names[c].split(" <- ")[1] in ("Lambda Lambda", "Sigma0 Sigma0")]
    assert len(same) == 10
    C = orc.correlator(L, F["u"][0], F["d"][0], F["s"][0], same)
    R = pj.project_spin(C)
    for i in range(len(same)):
        scale = np.abs(C[i]).max()
        assert scale > 0
        assert np.abs(R[i, :, 4:]).max() <= 1e-12 * scale
        assert np.abs(R[i, :, :4]).max() > 1e-3 * scale


# --------------------------------------------------------- cubic group
def test_cubic_rotations_form_the_rotation_group_of_the_cube():
    Rs = pj.cubic_rotations()
    assert len(Rs) == 24
    keys = {M.tobytes() for M in Rs}
    assert len(keys) == 24
    assert any((M == np.eye(3, dtype=np.int64)).all() for M in Rs)
    for A in Rs:
        assert (A @ A.T == np.eye(3)).all() and round(np.linalg.det(A)) == 1
        for B in Rs:
            assert (A @ B).tobytes() in keys
    # the rotations fixing the z axis are the four of C4
    assert sum(1 for M in Rs if (M[:, 2] == [0, 0, 1]).all()) == 4


def _coords(L):
    i = np.arange(L ** 3)
    return i % L, (i // L) % L, i // (L * L)


@pytest.mark.parametrize("L", [3, 4, 6])
def test_a1_closed_forms(L):
    x, y, z = _coords(L)
    c = lambda u: np.cos(2 * np.pi * u / L)
    s = lambda u: np.sin(2 * np.pi * u / L)
    inv = c(x) + c(y) + c(z) + 2 * c(x) * c(y) * c(z)
    assert np.allclose(pj.project_a1(inv[:, None], L)[:, 0], inv, atol=1e-14)
    for f in (s(x), s(y) * c(z), c(x) - c(y), c(x) + c(y) - 2 * c(z), s(x) * s(y)):
        assert np.abs(pj.project_a1(f[:, None], L)).max() < 1e-14
    # plane wave of momentum 2 pi / L along x: the orbit {+-e_i} averaged
    pw = np.exp(2j * np.pi * x / L)
    want = (c(x) + c(y) + c(z)) / 3
    assert np.allclose(pj.project_a1(pw[:, None], L)[:, 0], want, atol=1e-14)


def test_a1_is_a_projector_and_commutes_with_spin():
    L = 4
    rng = np.random.default_rng(9)
    F = rng.normal(size=(2, L ** 3, 16)) + 1j * rng.normal(size=(2, L ** 3, 16))
    P1 = pj.project_a1(F, L)
    assert np.allclose(pj.project_a1(P1, L), P1, atol=1e-13)
    Q1 = F - P1
    assert np.allclose(pj.project_a1(Q1, L), 0, atol=1e-13)
    assert np.allclose(pj.project_spin(P1), pj.project_a1(pj.project_spin(F), L), atol=1e-13)
    # the value at the origin is the plain average over nothing but itself
    assert np.allclose(P1[:, 0], F[:, 0], atol=1e-14)
