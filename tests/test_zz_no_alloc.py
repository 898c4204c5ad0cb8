"""The allocation-free IB forcing entry point (lbib_ib_force_noalloc) against
the simulation path (lbib_set_populations + lbib_read_ib_force) and the FP64
oracle.

Some callers cannot allocate device memory: solvers embedded in a host
application that owns every device allocation through its own arena, and
real-time loops that must not call an allocator once running.  They use this
call with their own device buffers; its only scratch is a static device array
shared by every call.  Two calls in a row with different particles and
populations must each match, so nothing left in the shared scratch by the
first call can leak into the second.  This file is named to run last in the
suite."""
import numpy as np
import pytest

from paper_1808_01448_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def eq_field(O, rho, ux, uy):
    ny, nx = rho.shape
    f = np.empty((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            f[:, y, x] = O.equilibrium(rho[y, x], ux[y, x], uy[y, x])
    return f


def case(O, seed, shape, xc, yc, theta, walls, ib_iterations=1):
    rng = np.random.default_rng(seed)
    nx, ny = 90, 48
    cfg = dict(nx=nx, ny=ny, wall_bottom=walls, wall_top=walls, tau=0.9,
               u_top=0.0 if walls == "periodic" else 0.02, ib_iterations=ib_iterations)
    rho = 1 + W.smooth_field(rng, nx, ny, 0.01)
    f = eq_field(O, rho, W.smooth_field(rng, nx, ny, 0.01), W.smooth_field(rng, nx, ny, 0.01))
    vx, vy = W.particle_outline(shape, 7.0)
    return cfg, f, dict(vx=vx, vy=vy, xc=xc, yc=yc, theta=theta)


def reference(L, cfg, f, part):
    s = L.Sim(storage="f32", **cfg)
    s.add_particle(ligand_density=0.0, sigma=0.0, **part)
    s.set_populations(f)
    fx, fy = s.ib_force()
    s.close()
    return fx, fy


def oracle_force(O, cfg, f, part):
    o = O.OracleSim(**cfg)
    o.add_particle(ligand_density=0.0, sigma=0.0, fixed=True, **part)
    o.set_populations(f)
    return o.ib_force()


def run_noalloc(torch, lbib, w, cfg, f, part, stream=None):
    ny, nx = cfg["ny"], cfg["nx"]
    dev = torch.tensor((f - w[:, None, None]).astype(np.float32), device="cuda")
    fx = torch.full((ny, nx), np.nan, dtype=torch.float64, device="cuda")
    fy = torch.full((ny, nx), np.nan, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    lbib.ib_force_noalloc(cfg, dev.data_ptr(), part["vx"], part["vy"], part["xc"],
                          part["yc"], part["theta"], fx_dev_ptr=fx.data_ptr(),
                          fy_dev_ptr=fy.data_ptr(),
                          stream=None if stream is None else stream.cuda_stream)
    torch.cuda.synchronize()
    return fx.cpu().numpy(), fy.cpu().numpy()


def test_noalloc_ib_force_matches_simulation_path_twice(O):
    torch = pytest.importorskip("torch")
    from paper_1808_01448_gb300 import build, lbib
    build.build()
    _, _, w, _ = O.lattice()
    side = torch.cuda.Stream()
    cases = [(case(O, 21, "ar2", 44.3, 17.6, 0.4, "bounce_back"), None),
             (case(O, 22, "circle", 20.7, 9.2, 0.0, "zou_he"), None),
             # multi-direct forcing on a caller-given stream
             (case(O, 23, "ar3", 51.2, 21.4, 1.1, "zou_he", ib_iterations=3), side)]
    for (cfg, f, part), stream in cases:
        gx, gy = run_noalloc(torch, lbib, w, cfg, f, part, stream)
        rx, ry = reference(lbib, cfg, f, part)
        scale = max(np.abs(rx).max(), np.abs(ry).max())
        assert scale > 1e-5
        np.testing.assert_allclose(gx, rx, rtol=0, atol=1e-6 * scale)
        np.testing.assert_allclose(gy, ry, rtol=0, atol=1e-6 * scale)
        # and the FP64 oracle (the FP32 path's inputs and arithmetic)
        ox, oy = oracle_force(O, cfg, f, part)
        np.testing.assert_allclose(gx, ox, rtol=0, atol=2e-6 * scale)
        np.testing.assert_allclose(gy, oy, rtol=0, atol=2e-6 * scale)


def test_noalloc_rejects_oversized_particle():
    from paper_1808_01448_gb300 import build, lbib
    build.build()
    # radius 100: the force tile alone (2 x 208^2 floats) exceeds the scratch;
    # the call fails before touching any device memory
    vx, vy = W.circle_polygon(100.0, 400)
    with pytest.raises(lbib.LbibError) as e:
        lbib.ib_force_noalloc(dict(nx=400, ny=300), 1, vx, vy, 200.0, 150.0,
                              fx_dev_ptr=1, fy_dev_ptr=1)
    assert e.value.status == "E_ARG"
    assert "scratch" in str(e.value)
