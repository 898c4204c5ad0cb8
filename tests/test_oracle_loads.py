"""Pins of the oracle's hydrodynamic loads (Eq. 7-8) against closed forms on
prescribed nodal fields.  Element geometry for the expected values is built
here from the vertices with numpy (midpoints, edge normals, shoelace area)."""
import math

import numpy as np
import pytest

from paper_1808_01448_gb300 import workloads as W


def geometry(vx, vy, xc, yc, th):
    c, s = math.cos(th), math.sin(th)
    X = xc + c * vx - s * vy
    Y = yc + s * vx + c * vy
    X2, Y2 = np.roll(X, -1), np.roll(Y, -1)
    dx, dy = X2 - X, Y2 - Y
    S = np.hypot(dx, dy)
    nx, ny = dy / S, -dx / S
    area = 0.5 * np.sum(X * Y2 - X2 * Y)
    return 0.5 * (X + X2), 0.5 * (Y + Y2), nx, ny, S, area


SHAPES = [("circle", 6.0, 0.0), ("ar2", 6.0, 0.3), ("ar3", 6.0, 1.1)]


def grid(c):
    y, x = np.mgrid[0:c.ny, 0:c.nx].astype(float)
    return x, y


@pytest.mark.parametrize("shape,r,th", SHAPES)
def test_uniform_state_gives_no_load(O, shape, r, th):
    c = O.make_config(nx=48, ny=40, tau=0.9)
    vx, vy = W.particle_outline(shape, r)
    rho = np.full((c.ny, c.nx), 1.003)
    z = np.zeros_like(rho)
    F = O.loads(c, rho, z, z, vx, vy, 24.2, 19.7, th)
    np.testing.assert_allclose(F, 0.0, atol=1e-14)


@pytest.mark.parametrize("shape,r,th", SHAPES)
@pytest.mark.parametrize("axis", [0, 1])
def test_linear_pressure_closed_form(O, shape, r, th, axis):
    """p = G x_axis is reproduced exactly by the linear MLS, so the discrete
    Eq. 7 with the 1.2 dx probe shift gives
    F_a = -G (A delta_ab + 1.2 sum n_a n_b S)."""
    c = O.make_config(nx=48, ny=40, tau=0.9)
    x, y = grid(c)
    G = 1e-4
    coord = x if axis == 0 else y
    rho = 1.0 + 3.0 * G * coord          # p = c_s^2 (rho - 1) = G coord
    z = np.zeros_like(rho)
    vx, vy = W.particle_outline(shape, r)
    xc, yc = 23.6, 19.2
    F = O.loads(c, rho, z, z, vx, vy, xc, yc, th)
    mx, my, nx, ny, S, A = geometry(vx, vy, xc, yc, th)
    na = nx if axis == 0 else ny
    expect = [-G * ((A if axis == 0 else 0.0) + 1.2 * np.sum(na * nx * S)),
              -G * ((A if axis == 1 else 0.0) + 1.2 * np.sum(na * ny * S))]
    assert F[0] == pytest.approx(expect[0], rel=1e-10, abs=1e-16)
    assert F[1] == pytest.approx(expect[1], rel=1e-10, abs=1e-16)


def test_linear_pressure_on_regular_polygon_has_no_moment(O):
    """Element centroids of a regular polygon lie along their own normals, so
    a pressure load has no moment about the centre."""
    c = O.make_config(nx=48, ny=40, tau=0.9)
    x, y = grid(c)
    vx, vy = W.circle_polygon(7.0, 44)
    rho = 1.0 + 3e-4 * x - 2e-4 * y
    z = np.zeros_like(rho)
    F = O.loads(c, rho, z, z, vx, vy, 24.0, 20.0, 0.37)
    assert abs(F[2]) < 1e-15
    assert abs(F[0]) > 1e-4


@pytest.mark.parametrize("shape,r,th", SHAPES)
def test_rigid_rotation_and_uniform_shear_give_no_load(O, shape, r, th):
    """Rigid rotation has no strain rate; a uniform shear has a constant
    symmetric stress whose resultant and moment on a closed outline vanish."""
    c = O.make_config(nx=48, ny=40, tau=0.9)
    x, y = grid(c)
    vx, vy = W.particle_outline(shape, r)
    xc, yc = 24.3, 19.9
    om = 2e-3
    rho = np.ones_like(x)
    F = O.loads(c, rho, -om * (y - yc), om * (x - xc), vx, vy, xc, yc, th)
    np.testing.assert_allclose(F, 0.0, atol=1e-16)
    gam = 1e-3
    F = O.loads(c, rho, gam * y, np.zeros_like(x), vx, vy, xc, yc, th)
    np.testing.assert_allclose(F, 0.0, atol=1e-15)


def test_viscous_traction_matches_newtonian_stress(O):
    """u = (a y^2, 0) has a linearly varying shear stress nu * 2 a y; the load
    on a circle is reproduced by summing nu (grad u + grad u^T) n S with the
    exact gradient at each probe (the MLS gradient of a quadratic field is
    exact at the node spacing only to O(h^2), so compare loosely)."""
    c = O.make_config(nx=64, ny=48, tau=0.8)
    x, y = grid(c)
    a = 1e-5
    vx, vy = W.circle_polygon(8.0, 50)
    xc, yc = 31.7, 23.4
    F = O.loads(c, np.ones_like(x), a * y * y, np.zeros_like(x), vx, vy, xc, yc, 0.0)
    mx, my, nx, ny, S, A = geometry(vx, vy, xc, yc, 0.0)
    qy = my + 1.2 * ny
    nu = (0.8 - 0.5) / 3
    txy = nu * 2 * a * qy
    Fx = np.sum(txy * ny * S)
    Fy = np.sum(txy * nx * S)
    assert F[0] == pytest.approx(Fx, rel=1e-3)
    assert abs(F[1] - Fy) < 1e-3 * abs(Fx)
