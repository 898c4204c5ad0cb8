"""Pins of the oracle's rigid-body update (Eq. 13-16) and of the coupled
step on flows whose outcome is known."""
import math

import numpy as np
import pytest

from paper_1808_01448_gb300 import workloads as W


def test_bdf2_velocity_closed_form(O):
    """Constant acceleration a from rest (u^{-1} = u^{-2} = 0): the recurrence
    3 u_n - 4 u_{n-1} + u_{n-2} = 2 a has the solution
    u_n = a (n + 1/2 + 3^{-n} / 6)."""
    a = 2.5e-4
    u1 = u2 = 0.0
    for n in range(40):
        u = O.bdf2_velocity(u1, u2, a)
        assert u == pytest.approx(a * (n + 0.5 + 3.0 ** (-n) / 6.0), rel=1e-13)
        u2, u1 = u1, u


def test_bdf2_position_closed_form(O):
    """Constant velocity U from x^{-1} = x^0: x_k = x_0 + U k - U/2 (1 - 3^{-k})."""
    x0, U = 3.0, 1e-3
    x1, x2 = x0, x0
    for k in range(1, 30):
        x = O.bdf2_position(x1, x2, U)
        assert x == pytest.approx(x0 + U * k - 0.5 * U * (1 - 3.0 ** (-k)), rel=1e-14)
        x2, x1 = x1, x


def test_particle_in_fluid_at_rest_stays_at_rest(O):
    s = O.OracleSim(nx=40, ny=30, tau=0.9)
    vx, vy = W.particle_outline("ar2", 5.0)
    s.add_particle(vx, vy, 20.0, 15.0, theta=0.4, ligand_density=0.0)
    s.step(50)
    p = s.particle(0)
    # loads, bond and wall forces vanish up to the rounding of sum_i w_i = 1
    np.testing.assert_allclose([p["u"], p["v"], p["omega"]], 0.0, atol=1e-14)
    np.testing.assert_allclose([*p["Fh"], p["Mh"]], 0.0, atol=1e-13)
    np.testing.assert_allclose([p["xc"], p["yc"], p["theta"]], [20.0, 15.0, 0.4], rtol=1e-13)


def test_polygon_mass_properties(O):
    s = O.OracleSim(nx=60, ny=50)
    vx, vy = W.ellipse_polygon(6.0, 12.0, 400)
    s.add_particle(vx, vy, 30.0, 25.0, rho_p=1.3)
    p = s.particle(0)
    A = math.pi * 6 * 12
    assert p["area"] == pytest.approx(A, rel=1e-3)
    assert p["mass"] == pytest.approx(1.3 * p["area"], rel=1e-15)
    assert p["inertia"] == pytest.approx(1.3 * A * (36 + 144) / 4, rel=2e-3)
    assert p["r_eq"] == pytest.approx(math.sqrt(72), rel=1e-3)


def test_free_circle_in_shear_rotates_at_half_the_shear_rate(O):
    """A neutrally buoyant free circle at mid-channel in simple shear turns at
    Omega ~ gamma / 2 (Stokes-flow value; confinement and the diffuse
    interface allow a few per cent)."""
    nx, ny, umax = 64, 33, 0.01
    cfg = dict(nx=nx, ny=ny, wall_bottom="zou_he", wall_top="zou_he", tau=1.0, u_top=umax)
    s = O.OracleSim(**cfg)
    ex, ey, w, _ = O.lattice()
    yy = np.arange(ny)[:, None] * np.ones((1, nx))
    f = np.empty((9, ny, nx))
    for y in range(ny):
        feq = O.equilibrium(1.0, umax * y / (ny - 1), 0.0)
        f[:, y, :] = feq[:, None]
    s.set_populations(f)
    vx, vy = W.circle_polygon(5.0, 31)
    s.add_particle(vx, vy, 32.0, 16.0, ligand_density=0.0)
    s.step(2500)
    p = s.particle(0)
    gamma = umax / (ny - 1)
    assert p["omega"] == pytest.approx(-gamma / 2, rel=0.15)
    assert abs(p["yc"] - 16.0) < 0.05
    assert p["u"] == pytest.approx(umax * 16.0 / (ny - 1), rel=0.05)
