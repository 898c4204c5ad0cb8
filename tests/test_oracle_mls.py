"""Pins of the oracle's moving-least-squares interpolation and spreading
(Sec. 'The combined LB-IB method', refs [13], [39]): properties of the
B-spline weight, partition of unity, linear reproduction, exact gradients of
linear fields, a brute-force weighted least-squares fit, and the adjoint
relation between interpolation and spreading."""
import numpy as np
import pytest


def test_weight_is_cubic_bspline(O):
    """Integer translates of the cubic B-spline sum to one, have zero first
    moment and second moment 1/3; the kernel is even, non-negative and
    supported on |r| < 2."""
    rng = np.random.default_rng(3)
    for x in rng.uniform(-3, 3, 50):
        ks = np.arange(int(np.floor(x)) - 3, int(np.floor(x)) + 4)
        w = np.array([O.weight(k - x) for k in ks])
        assert w.sum() == pytest.approx(1.0, abs=1e-15)
        assert (w * (ks - x)).sum() == pytest.approx(0.0, abs=1e-15)
        assert (w * (ks - x) ** 2).sum() == pytest.approx(1.0 / 3.0, abs=1e-14)
        assert np.all(w >= 0)
    assert O.weight(0.0) == pytest.approx(2.0 / 3.0, abs=1e-16)
    assert O.weight(2.0) == 0.0 and O.weight(-2.5) == 0.0
    assert O.weight(0.7) == O.weight(-0.7)


def cfg(O, **kw):
    base = dict(nx=40, ny=24, wall_bottom="bounce_back", wall_top="bounce_back")
    base.update(kw)
    return O.make_config(**base)


def unwrap(ix, X, nx):
    """Node x coordinate nearest to X (undo the periodic wrap)."""
    return ix + nx * np.round((X - ix) / nx)


@pytest.mark.parametrize("walls", ["bounce_back", "zou_he", "periodic"])
def test_partition_of_unity_and_linear_reproduction(O, walls):
    c = cfg(O, wall_bottom=walls, wall_top=walls)
    rng = np.random.default_rng(4)
    pts = [(rng.uniform(-3, 43), rng.uniform(0.3, 22.7)) for _ in range(200)]
    pts += [(5.0, 7.0), (0.0, 1.0), (39.9, 3.5), (12.5, 22.9)]
    for X, Y in pts:
        ix, iy, phi = O.mls_shape(c, X, Y)
        assert len(phi) > 0
        xk = unwrap(ix, X, c.nx)
        yk = iy.astype(float)
        if walls == "periodic":
            yk = unwrap(iy, Y, c.ny)
        assert phi.sum() == pytest.approx(1.0, abs=1e-13)
        assert (phi * xk).sum() == pytest.approx(X, abs=1e-12)
        assert (phi * yk).sum() == pytest.approx(Y, abs=1e-12)


def test_support_respects_walls(O):
    """Only lattice rows enter the support (wall nodes included, so a point
    between the wall row and row 1 is inside its support's row span); a point
    beyond a wall line (y = 0 and ny - 1 for Zou-He, -1/2 and ny - 1/2 for
    bounce-back) has no fit."""
    for walls, yb, yt in (("zou_he", 0.0, 23.0), ("bounce_back", -0.5, 23.5)):
        c = cfg(O, wall_bottom=walls, wall_top=walls)
        ix, iy, phi = O.mls_shape(c, 10.3, 0.4)
        assert iy.min() == 0 and iy.max() == 2
        assert np.all(phi > -1e-12)                       # no extrapolation weights
        _, iy, _ = O.mls_shape(c, 10.3, c.ny - 1.4)
        assert iy.max() == c.ny - 1
        assert len(O.mls_shape(c, 10.3, yb)[2]) > 0       # on the wall line
        assert len(O.mls_shape(c, 10.3, yt)[2]) > 0
        assert len(O.mls_shape(c, 10.3, yb - 1e-9)[2]) == 0
        assert len(O.mls_shape(c, 10.3, yt + 1e-9)[2]) == 0
        assert len(O.mls_shape(c, 10.3, -1.9)[2]) == 0


def test_fit_is_well_conditioned_up_to_the_walls(O):
    """Everywhere in the fluid, wall lines included, the shape functions stay
    bounded (no near-singular extrapolation from one usable row) and still
    reproduce linear fields."""
    for walls, yb, yt in (("zou_he", 0.0, 23.0), ("bounce_back", -0.5, 23.5)):
        c = cfg(O, wall_bottom=walls, wall_top=walls)
        for Y in np.concatenate([np.linspace(yb, yb + 2.0, 81), np.linspace(yt - 2.0, yt, 81)]):
            ix, iy, phi = O.mls_shape(c, 17.37, Y)
            assert len(phi) > 0
            assert np.abs(phi).max() < 1.5
            assert phi.sum() == pytest.approx(1.0, abs=1e-12)
            assert (phi * iy).sum() == pytest.approx(Y, abs=1e-11)


def test_fit_is_exact_on_linear_fields(O):
    c = cfg(O)
    y, x = np.mgrid[0:c.ny, 0:c.nx].astype(float)
    field = 0.3 + 0.02 * x - 0.05 * y
    rng = np.random.default_rng(5)
    for _ in range(100):
        X, Y = rng.uniform(3, 36), rng.uniform(0.2, 22.8)
        n, v, dx, dy = O.mls_fit(c, field, X, Y)
        assert n > 0
        assert v == pytest.approx(0.3 + 0.02 * X - 0.05 * Y, abs=1e-13)
        assert dx == pytest.approx(0.02, abs=1e-13)
        assert dy == pytest.approx(-0.05, abs=1e-13)


def test_fit_matches_brute_force_weighted_least_squares(O):
    """Independent solve: numpy lstsq of the sqrt(w)-scaled basis over the
    same support, with the separately pinned B-spline weight."""
    c = cfg(O, wall_bottom="zou_he", wall_top="zou_he")
    rng = np.random.default_rng(6)
    field = rng.normal(size=(c.ny, c.nx))
    for _ in range(60):
        X, Y = rng.uniform(0, 40), rng.uniform(0.5, 22.5)
        ix, iy, phi = O.mls_shape(c, X, Y)
        xk = unwrap(ix, X, c.nx)
        dx, dy = xk - X, iy - Y
        w = np.array([O.weight(a) * O.weight(b) for a, b in zip(dx, dy)])
        P = np.stack([np.ones_like(dx), dx, dy], axis=1)
        s = np.sqrt(w)
        coef, *_ = np.linalg.lstsq(P * s[:, None], field[iy, ix] * s, rcond=None)
        n, v, gx, gy = O.mls_fit(c, field, X, Y)
        assert v == pytest.approx(coef[0], abs=1e-12)
        assert gx == pytest.approx(coef[1], abs=1e-12)
        assert gy == pytest.approx(coef[2], abs=1e-12)
        assert (phi * field[iy, ix]).sum() == pytest.approx(coef[0], abs=1e-12)


def test_periodic_wrap_in_x(O):
    c = cfg(O)
    rng = np.random.default_rng(7)
    field = rng.normal(size=(c.ny, c.nx))
    shifted = np.roll(field, 5, axis=1)
    for X in (0.2, 1.7, 38.9, 39.99):
        a = O.mls_fit(c, field, X, 9.3)
        b = O.mls_fit(c, shifted, X + 5, 9.3)
        assert a[1] == pytest.approx(b[1], abs=1e-13)


def test_spreading_conserves_force_and_is_adjoint(O):
    c = cfg(O)
    rng = np.random.default_rng(8)
    n = 30
    t = np.linspace(0, 2 * np.pi, n, endpoint=False)
    X, Y = 20 + 6 * np.cos(t), 11 + 6 * np.sin(t)
    Fx, Fy, eps = rng.normal(size=n), rng.normal(size=n), rng.uniform(0.8, 1.2, n)
    fx, fy = O.spread(c, X, Y, Fx, Fy, eps)
    assert fx.sum() == pytest.approx((Fx * eps).sum(), abs=1e-12)
    assert fy.sum() == pytest.approx((Fy * eps).sum(), abs=1e-12)
    u = rng.normal(size=(c.ny, c.nx))
    lhs = (eps * Fx * O.interp(c, u, X, Y)).sum()
    assert lhs == pytest.approx((u * fx).sum(), abs=1e-12)
    # interpolating a constant returns it (partition of unity)
    np.testing.assert_allclose(O.interp(c, np.full((c.ny, c.nx), 2.5), X, Y), 2.5, atol=1e-13)


def test_multi_direct_forcing_reduces_slip(O):
    """Multi-direct forcing: with each added pass the velocity at the markers,
    after the final force is spread, comes closer to the rigid motion (here a
    fixed particle in a sheared, perturbed flow, so the target is zero); the
    single pass leaves a slip of the order of the local flow."""
    from paper_1808_01448_gb300 import workloads as W
    nx, ny = 96, 48
    f = np.zeros((9, ny, nx))
    for j in range(ny):
        for i in range(nx):
            f[:, j, i] = O.equilibrium(1.0, 0.03 * (j + 0.5) / ny,
                                       0.004 * np.sin(2 * np.pi * i / nx))
    vx, vy = W.circle_polygon(8.0, 50)
    X, Y, *_ = O.elements(vx, vy, 48.3, 24.2, 0.0)
    slip = []
    for M in (1, 2, 3, 4):
        c = dict(nx=nx, ny=ny, wall_bottom="zou_he", wall_top="zou_he", tau=0.9, u_top=0.03,
                 ib_iterations=M)
        s = O.OracleSim(**c)
        s.add_particle(vx, vy, xc=48.3, yc=24.2, fixed=True)
        s.set_populations(f)
        _, u, v = s.fields()        # velocity with the spread force included
        cfg_ = O.make_config(**c)
        ul, vl = O.interp(cfg_, u, X, Y), O.interp(cfg_, v, X, Y)
        slip.append(np.sqrt(np.mean(ul ** 2 + vl ** 2)))
    assert slip[0] > 1e-3
    assert slip[0] > slip[1] > slip[2] > slip[3]
    assert slip[3] < 0.25 * slip[0]
