"""Pins of the oracle's solved spreading scales (Vanella & Balaras, ref. [39]
of Sec. "The combined LB-IB method"): sum_m A_lm eps_m = 1 with
A_lm = sum_k phi_k(X_l) phi_k(X_m).

 - A straight line of markers one node apart in a periodic lattice, away
   from the walls: every support is a full 4 x 4 one, the shape functions are
   the tensor B-spline weights, and A 1 = sum_j w(Y - y_j)^2 1 by the
   B-spline's partition of unity along x, so eps = 1 / sum_j w(Y - y_j)^2
   exactly at every marker.
 - A closed outline: the residual of A eps = 1 (A built here from the pinned
   shape functions) and the defining property -- interpolating the spread of
   a uniform marker force returns that force at every marker.
 - A coupled IB step in a uniform flow at rest particle: the Guo half-step
   velocity change interpolated at each marker is exactly -u0."""
import math

import numpy as np
import pytest

from paper_1808_01448_gb300 import workloads as W


def marker_line(nx, Y, x0):
    X = x0 + np.arange(nx, dtype=float)
    return X, np.full(nx, Y)


@pytest.mark.parametrize("Y,x0", [(11.37, 0.23), (9.81, 0.61), (12.0, 0.05)])
def test_straight_line_closed_form(O, Y, x0):
    nx = 16
    c = O.make_config(nx=nx, ny=24, wall_bottom="periodic", wall_top="periodic")
    X, Yv = marker_line(nx, Y, x0)
    eps = O.vb_eps(c, X, Yv)
    rows = np.arange(math.floor(Y) - 1, math.floor(Y) + 3)
    s2 = sum(O.weight(Y - y) ** 2 for y in rows)
    np.testing.assert_allclose(eps, 1.0 / s2, rtol=1e-11)


def outline_markers(shape, r, xc, yc, theta):
    vx, vy = W.particle_outline(shape, r)
    c, s = math.cos(theta), math.sin(theta)
    ax = xc + c * vx - s * vy
    ay = yc + s * vx + c * vy
    return 0.5 * (ax + np.roll(ax, -1)), 0.5 * (ay + np.roll(ay, -1))


def matrix(O, c, X, Y):
    sup = []
    for x, y in zip(X, Y):
        ix, iy, phi = O.mls_shape(c, x, y)
        sup.append({(int(a), int(b)): p for a, b, p in zip(ix, iy, phi)})
    n = len(X)
    A = np.zeros((n, n))
    for l in range(n):
        for m in range(n):
            A[l, m] = sum(v * sup[m].get(k, 0.0) for k, v in sup[l].items())
    return A


@pytest.mark.parametrize("walls,shape,yc", [("bounce_back", "circle", 20.3),
                                           ("zou_he", "ar3", 9.4),
                                           ("periodic", "ar2", 1.7)])
def test_system_residual_and_uniform_force_round_trip(O, walls, shape, yc):
    c = O.make_config(nx=64, ny=40, wall_bottom=walls, wall_top=walls)
    X, Y = outline_markers(shape, 6.0, 31.4, yc, 0.41)
    eps = O.vb_eps(c, X, Y)
    A = matrix(O, c, X, Y)
    # markers beyond a wall line have no fit: no row in A, eps = 0
    fit = np.array([len(O.mls_shape(c, x, y)[2]) > 0 for x, y in zip(X, Y)])
    assert fit.sum() >= len(X) - 4
    np.testing.assert_array_equal(eps[~fit], 0.0)
    np.testing.assert_allclose((A @ eps)[fit], 1.0, rtol=0, atol=1e-11)
    assert eps[fit].min() > 0.5 and eps.max() < 6.0
    F = np.full(len(X), 0.37)
    fx, fy = O.spread(c, X, Y, F, -F, eps)
    np.testing.assert_allclose(O.interp(c, fx, X, Y)[fit], F[fit], rtol=0, atol=1e-12)
    np.testing.assert_allclose(O.interp(c, fy, X, Y)[fit], -F[fit], rtol=0, atol=1e-12)


def test_ib_step_enforces_the_marker_velocity(O):
    """With the solved scales, one direct-forcing pass cancels a uniform slip
    exactly: F_l = 2 rho (U^d_l - u0) is uniform, so the interpolated Guo
    correction I_l[f_ib] / (2 rho) equals U^d_l - u0 = -u0 at every marker
    (with eps_l = S_l it is only about half of that)."""
    nx = ny = 48
    u0 = np.array([2e-3, 7e-4])
    cfg = dict(nx=nx, ny=ny, wall_bottom="periodic", wall_top="periodic", tau=0.9, ib_spread=1)
    f = np.broadcast_to(O.equilibrium(1.0, u0[0], u0[1])[:, None, None], (9, ny, nx)).copy()
    vx, vy = W.particle_outline("circle", 6.0)
    s = O.OracleSim(**cfg)
    s.add_particle(vx, vy, 23.7, 24.2, theta=0.3, ligand_density=0.0, sigma=0.0, fixed=True)
    s.set_populations(f)
    fx, fy = s.ib_force()
    X, Y = outline_markers("circle", 6.0, 23.7, 24.2, 0.3)
    c = O.make_config(**cfg)
    np.testing.assert_allclose(O.interp(c, fx, X, Y) / 2.0, -u0[0], rtol=1e-10)
    np.testing.assert_allclose(O.interp(c, fy, X, Y) / 2.0, -u0[1], rtol=1e-10)
    s1 = O.OracleSim(**dict(cfg, ib_spread=0))
    s1.add_particle(vx, vy, 23.7, 24.2, theta=0.3, ligand_density=0.0, sigma=0.0, fixed=True)
    s1.set_populations(f)
    g = O.interp(c, s1.ib_force()[0], X, Y) / 2.0 / -u0[0]
    assert 0.3 < g.mean() < 0.7
