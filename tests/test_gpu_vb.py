"""The solved spreading scales (ib_spread = 1, Vanella & Balaras, ref. [39] of
Sec. "The combined LB-IB method") on the GPU against the FP64 oracle's dense
solve of A eps = 1.

FP64 storage solves the cyclic-banded system in FP64 (bordered L D L^T), so
the IB force field agrees with the oracle's to rounding (1e-12 of its
scale).  FP32 storage solves it in FP32: A is built from FP32 shape
functions and its condition number reaches ~10^2, so the field agrees to
~1e-5 of its scale.  Coupled FP64 steps with the solved scales keep the bond
flags equal at every step."""
import numpy as np
import pytest

from paper_1808_01448_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1808_01448_gb300 import build, lbib
    build.build()
    return lbib


def eq_field(O, rho, ux, uy):
    ny, nx = rho.shape
    f = np.empty((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            f[:, y, x] = O.equilibrium(rho[y, x], ux[y, x], uy[y, x])
    return f


def start(O, nx, ny, seed, amp=0.01):
    rng = np.random.default_rng(seed)
    rho = 1 + W.smooth_field(rng, nx, ny, 0.01)
    return eq_field(O, rho, W.smooth_field(rng, nx, ny, amp), W.smooth_field(rng, nx, ny, amp))


def ib_pair(O, L, cfg, p, f0, storage):
    o = O.OracleSim(**cfg)
    o.add_particle(**p)
    o.set_populations(f0)
    g = L.Sim(storage=storage, **cfg)
    g.add_particle(**p)
    g.set_populations(f0)
    return o.ib_force(), g.ib_force(), g


@pytest.mark.parametrize("walls", ["bounce_back", "zou_he", "periodic"])
@pytest.mark.parametrize("shape,r", [("circle", 7.0), ("ar3", 10.0), ("circle", 20.0)])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_solved_scales_ib_force_parity(O, L, walls, shape, r, storage):
    nx, ny = 96, 64
    cfg = dict(nx=nx, ny=ny, wall_bottom=walls, wall_top=walls, tau=0.9,
               u_top=0.0 if walls == "periodic" else 0.02, ib_spread=1)
    f0 = start(O, nx, ny, 7)
    vx, vy = W.particle_outline(shape, r)
    yc = 2.7 if walls == "periodic" else (r * 1.8 if shape == "ar3" else r + 1.3)
    p = dict(vx=vx, vy=vy, xc=47.3, yc=yc, theta=0.35, ligand_density=0.0, sigma=0.0)
    fo, fg, g = ib_pair(O, L, cfg, p, f0, storage)
    scale = max(np.abs(fo[0]).max(), np.abs(fo[1]).max())
    assert scale > 1e-4
    tol = 1e-12 if storage == "f64" else 3e-5
    np.testing.assert_allclose(fg[0], fo[0], rtol=0, atol=tol * scale)
    np.testing.assert_allclose(fg[1], fo[1], rtol=0, atol=tol * scale)
    # the solved scales change the field (against eps_l = S_l)
    _, f1, g1 = ib_pair(O, L, dict(cfg, ib_spread=0), p, f0, storage)
    assert np.abs(f1[0] - fg[0]).max() > 0.1 * scale
    g.close()
    g1.close()


def test_solved_scales_with_multi_direct_forcing_f64(O, L):
    nx, ny = 80, 48
    cfg = dict(nx=nx, ny=ny, wall_bottom="zou_he", wall_top="zou_he", tau=0.9, u_top=0.02,
               ib_spread=1, ib_iterations=3)
    f0 = start(O, nx, ny, 8)
    vx, vy = W.particle_outline("ar2", 8.0)
    p = dict(vx=vx, vy=vy, xc=40.6, yc=16.3, theta=0.2, ligand_density=0.0, sigma=0.0)
    fo, fg, g = ib_pair(O, L, cfg, p, f0, "f64")
    scale = max(np.abs(fo[0]).max(), np.abs(fo[1]).max())
    np.testing.assert_allclose(fg[0], fo[0], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(fg[1], fo[1], rtol=0, atol=1e-12 * scale)
    g.close()


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_solved_scales_full_step(O, L, storage):
    """Coupled steps with the solved scales: FP64 to rounding with the bond
    flags equal at every step; FP32 within the FP32 tolerances."""
    cfg = W.shear_channel(112, 48, 1.0, tau=0.9, k_f=0.85, k_r0=0.03, kBT=0.02, seed=6,
                          sim_id=1, hamaker=1e-6, ib_spread=1)
    cfg["y_cr"] = 1.0
    p = W.adhesion_particle(cfg, "circle", 7.0, x=40.0, ligand_density=0.7, sigma=0.02,
                            gap_over_h=0.3 / 47)
    o = O.OracleSim(**cfg)
    o.add_particle(**p)
    g = L.Sim(storage=storage, **cfg)
    g.add_particle(**p)
    for t in range(80):
        o.step(1)
        g.step(1)
        if storage == "f64":
            assert np.array_equal(o.bonds(0)[0], g.bonds(0)[0]), f"step {t + 1}"
    po, pg = o.particle(0), g.particle(0)
    _, uo, vo = o.fields()
    _, ug, vg = g.fields()
    err = np.linalg.norm(np.stack([ug - uo, vg - vo])) / np.linalg.norm(np.stack([uo, vo]))
    if storage == "f64":
        assert err < 1e-11
        for k in ("xc", "yc", "theta", "u", "v", "omega"):
            assert pg[k] == pytest.approx(po[k], abs=1e-10), k
    else:
        assert err < 1e-5
        for k in ("xc", "yc", "theta"):
            assert abs(pg[k] - po[k]) < 1e-4, k
    g.close()


def test_too_thin_particle_is_refused(L):
    s = L.Sim(nx=96, ny=48, ib_spread=1)
    vx, vy = W.particle_outline("ar3", 4.0)      # tips fold within 4 sqrt 2
    with pytest.raises(L.LbibError) as e:
        s.add_particle(vx, vy, xc=40.0, yc=20.0)
    assert e.value.status == "E_ARG"
    vx, vy = W.particle_outline("ar3", 10.0)
    s.add_particle(vx, vy, xc=40.0, yc=20.0)
    s.step(2)
    s.synchronize()
    s.close()
