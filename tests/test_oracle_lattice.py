"""Pins of the oracle's lattice building blocks (Eq. 1-6) against moment
identities of the D2Q9 Hermite discretisation and Guo's forcing scheme."""
import numpy as np
import pytest

CS2 = 1.0 / 3.0


def test_lattice_tables_moments(O):
    ex, ey, w, opp = O.lattice()
    # Eq. 3 directions: unit speeds at i = 1..4, diagonals at 5..8
    speeds = ex ** 2 + ey ** 2
    assert list(speeds) == [0, 1, 1, 1, 1, 2, 2, 2, 2]
    assert np.all(ex[opp] == -ex) and np.all(ey[opp] == -ey)
    # weights: normalised, zero first moment, isotropic second moment c_s^2 I,
    # isotropic fourth moment (the properties that make Eq. 2 a Hermite projection)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert abs((w * ex).sum()) < 1e-15 and abs((w * ey).sum()) < 1e-15
    assert (w * ex * ex).sum() == pytest.approx(CS2, abs=1e-15)
    assert (w * ey * ey).sum() == pytest.approx(CS2, abs=1e-15)
    assert abs((w * ex * ey).sum()) < 1e-15
    assert (w * ex ** 4).sum() == pytest.approx(3 * CS2 ** 2, abs=1e-15)
    assert (w * ex ** 2 * ey ** 2).sum() == pytest.approx(CS2 ** 2, abs=1e-15)


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.02, 0.03, -0.01),
                                       (0.97, -0.05, 0.04)])
def test_equilibrium_moments(O, rho, ux, uy):
    """Eq. 2 reproduces rho, rho u and the Euler stress rho (c_s^2 I + u u)."""
    ex, ey, w, _ = O.lattice()
    f = O.equilibrium(rho, ux, uy)
    assert f.sum() == pytest.approx(rho, rel=1e-14)
    assert (f * ex).sum() == pytest.approx(rho * ux, abs=1e-15)
    assert (f * ey).sum() == pytest.approx(rho * uy, abs=1e-15)
    assert (f * ex * ex).sum() == pytest.approx(rho * (CS2 + ux * ux), rel=1e-14)
    assert (f * ey * ey).sum() == pytest.approx(rho * (CS2 + uy * uy), rel=1e-14)
    assert (f * ex * ey).sum() == pytest.approx(rho * ux * uy, abs=1e-15)


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0, 1.7])
def test_guo_source_moments(O, tau):
    """Guo et al. (2002): sum F_i = 0, sum F_i e_i = (1 - 1/2tau) F,
    sum F_i e_i e_i = (1 - 1/2tau)(u F + F u)."""
    ex, ey, w, _ = O.lattice()
    ux, uy, Fx, Fy = 0.02, -0.03, 1e-3, 2e-3
    S = O.guo_source(tau, ux, uy, Fx, Fy)
    k = 1.0 - 0.5 / tau
    assert abs(S.sum()) < 1e-17
    assert (S * ex).sum() == pytest.approx(k * Fx, rel=1e-13)
    assert (S * ey).sum() == pytest.approx(k * Fy, rel=1e-13)
    assert (S * ex * ex).sum() == pytest.approx(k * 2 * ux * Fx, rel=1e-12)
    assert (S * ey * ey).sum() == pytest.approx(k * 2 * uy * Fy, rel=1e-12)
    assert (S * ex * ey).sum() == pytest.approx(k * (ux * Fy + uy * Fx), rel=1e-12)


def test_collision_conserves_mass_and_adds_force(O):
    """BGK with Guo forcing and the half-force velocity of Eq. 6: mass is
    conserved and the momentum grows by exactly F per step."""
    rng = np.random.default_rng(0)
    ex, ey, w, _ = O.lattice()
    for tau in (0.55, 0.8, 1.3):
        f = O.equilibrium(1.01, 0.02, -0.01) * (1 + 0.01 * rng.uniform(-1, 1, 9))
        Fx, Fy = 3e-4, -1e-4
        g = O.collide_node(f, tau, Fx, Fy)
        assert g.sum() == pytest.approx(f.sum(), rel=1e-15)
        assert (g * ex).sum() - (f * ex).sum() == pytest.approx(Fx, rel=1e-10)
        assert (g * ey).sum() - (f * ey).sum() == pytest.approx(Fy, rel=1e-10)


def test_collision_relaxes_non_equilibrium_by_one_minus_inverse_tau(O):
    """Without force, the non-equilibrium part is scaled by (1 - 1/tau)."""
    ex, ey, w, _ = O.lattice()
    feq = O.equilibrium(1.0, 0.01, 0.02)
    neq = np.array([0, 1, -1, 1, -1, 0.5, -0.5, 0.5, -0.5]) * 1e-4  # zero mass/momentum
    assert abs(neq.sum()) < 1e-18 and abs((neq * ex).sum()) < 1e-18
    assert abs((neq * ey).sum()) < 1e-18
    tau = 0.7
    g = O.collide_node(feq + neq, tau, 0.0, 0.0)
    np.testing.assert_allclose(g - feq, (1 - 1 / tau) * neq, atol=1e-15)
