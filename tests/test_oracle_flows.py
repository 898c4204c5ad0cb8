"""Pins of the oracle's fluid step (Eq. 1-6, walls) against flows with closed
forms and exact conservation laws."""
import math

import numpy as np
import pytest


def eq_field(O, rho, ux, uy):
    """f = f^eq(rho, u) at every node, [9][ny][nx] (the oracle's Eq. 2)."""
    ny, nx = rho.shape
    f = np.empty((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            f[:, y, x] = O.equilibrium(rho[y, x], ux[y, x], uy[y, x])
    return f


def total_momentum(O, f):
    ex, ey, _, _ = O.lattice()
    return (f * ex[:, None, None]).sum(), (f * ey[:, None, None]).sum()


def test_rest_state_is_a_fixed_point(O):
    """f^eq(1, 0) is a fixed point of collide + stream for every wall kind
    (to the rounding of the weights)."""
    for walls in ("bounce_back", "zou_he", "periodic"):
        s = O.OracleSim(nx=12, ny=8, wall_bottom=walls, wall_top=walls, tau=0.9)
        f0 = s.populations()
        s.step(25)
        np.testing.assert_allclose(s.populations(), f0, rtol=0, atol=4e-16)


@pytest.mark.parametrize("walls", ["bounce_back", "periodic"])
def test_mass_is_conserved(O, walls):
    rng = np.random.default_rng(1)
    nx, ny = 16, 10
    s = O.OracleSim(nx=nx, ny=ny, wall_bottom=walls, wall_top=walls, tau=0.7,
                    u_top=0.02 if walls == "bounce_back" else 0.0, gx=1e-5)
    rho = 1 + 0.01 * rng.uniform(-1, 1, (ny, nx))
    f = eq_field(O, rho, 0.01 * rng.uniform(-1, 1, (ny, nx)), 0.01 * rng.uniform(-1, 1, (ny, nx)))
    s.set_populations(f)
    m0 = f.sum()
    s.step(50)
    assert s.populations().sum() == pytest.approx(m0, rel=1e-14)


def test_periodic_box_momentum_grows_by_body_force(O):
    """Guo forcing in a fully periodic box: total momentum of f* grows by
    exactly N g per step."""
    rng = np.random.default_rng(2)
    nx, ny, gx, gy = 12, 10, 2e-6, -1e-6
    s = O.OracleSim(nx=nx, ny=ny, wall_bottom="periodic", wall_top="periodic", tau=0.8,
                    gx=gx, gy=gy)
    rho = 1 + 0.005 * rng.uniform(-1, 1, (ny, nx))
    f = eq_field(O, rho, 0.01 * rng.uniform(-1, 1, (ny, nx)), np.zeros((ny, nx)))
    s.set_populations(f)
    px0, py0 = total_momentum(O, f)
    n = 40
    s.step(n)
    px, py = total_momentum(O, s.populations())
    assert px - px0 == pytest.approx(n * nx * ny * gx, rel=1e-9)
    assert py - py0 == pytest.approx(n * nx * ny * gy, rel=1e-9)


@pytest.mark.parametrize("walls", ["zou_he", "bounce_back"])
def test_couette_linear_profile(O, walls):
    """Wall-driven shear (Sec. 'Modeling the adhesion dynamics'): the steady
    state is u_x = u_max (y - y_b) / H with the wall lines at rows 0 and ny-1
    (Zou-He) or half a spacing outside (bounce-back)."""
    nx, ny, umax = 8, 17, 1e-3
    s = O.OracleSim(nx=nx, ny=ny, wall_bottom=walls, wall_top=walls, tau=1.0, u_top=umax)
    y = np.arange(ny, dtype=float)
    if walls == "zou_he":
        prof = umax * y / (ny - 1)
    else:
        prof = umax * (y + 0.5) / ny
    s.step(6000)
    rho, ux, uy = s.fields()
    np.testing.assert_allclose(ux, np.broadcast_to(prof[:, None], ux.shape), atol=1e-12 * 1e3 * umax)
    assert np.abs(uy).max() < 1e-14
    np.testing.assert_allclose(rho, 1.0, atol=1e-12)


def poiseuille(O, tau, ny=16, steps=None):
    nx, g = 8, 1e-6
    nu = (tau - 0.5) / 3
    s = O.OracleSim(nx=nx, ny=ny, wall_bottom="bounce_back", wall_top="bounce_back",
                    tau=tau, gx=g)
    steps = steps or int(40 * ny * ny / nu / math.pi ** 2)
    s.step(steps)
    rho, ux, uy = s.fields()
    return ux[:, 0], g, nu, ny


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2])
def test_poiseuille_bulk_is_exact_parabola(O, tau):
    """Body-force Poiseuille flow between half-way bounce-back walls: in the
    bulk the steady LB solution satisfies nu u'' = -g exactly."""
    u, g, nu, ny = poiseuille(O, tau)
    d2 = u[2:] - 2 * u[1:-1] + u[:-2]
    np.testing.assert_allclose(nu * d2, -g, rtol=1e-8)


def test_poiseuille_magic_tau_has_no_slip(O):
    """For BGK with half-way bounce-back the wall sits exactly halfway when
    tau = 1/2 + sqrt(3/16) (He, Zou, Luo, Dembo 1997): the profile equals
    g/(2 nu) (y + 1/2)(H - 1/2 - y), H = ny."""
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    u, g, nu, ny = poiseuille(O, tau)
    y = np.arange(ny)
    exact = g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    np.testing.assert_allclose(u, exact, rtol=1e-8)
    # and away from it the slip is visible (the pin is not vacuous)
    u2, g2, nu2, _ = poiseuille(O, 1.2)
    exact2 = g2 / (2 * nu2) * (y + 0.5) * (ny - 0.5 - y)
    assert abs(u2[0] - exact2[0]) > 1e-3 * exact2[0]


def taylor_green_rate(O, N, tau, U=1e-4, t1=50, t2=250):
    nu = (tau - 0.5) / 3
    k = 2 * math.pi / N
    x = np.arange(N)[None, :].astype(float)
    y = np.arange(N)[:, None].astype(float)
    ux = -U * np.cos(k * x) * np.sin(k * y)
    uy = U * np.sin(k * x) * np.cos(k * y)
    s = O.OracleSim(nx=N, ny=N, wall_bottom="periodic", wall_top="periodic", tau=tau)
    s.set_populations(eq_field(O, np.ones((N, N)), ux, uy))
    s.step(t1)
    a1 = np.abs(s.fields()[1]).max()
    s.step(t2 - t1)
    a2 = np.abs(s.fields()[1]).max()
    rate = math.log(a1 / a2) / (t2 - t1)
    return rate, 2 * nu * k * k


def test_taylor_green_decay_checks_viscosity(O):
    """A decaying Taylor-Green vortex decays as exp(-2 nu k^2 t) with
    nu = (tau - 1/2)/3; the lattice error shrinks at second order."""
    errs = []
    for N in (16, 32):
        rate, exact = taylor_green_rate(O, N, tau=0.8)
        errs.append(abs(rate / exact - 1))
    assert errs[1] < 5e-3
    assert errs[0] / errs[1] > 3.0
