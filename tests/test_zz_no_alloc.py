"""The allocation-free IB forcing entry point (lbib_ib_force_noalloc) against
the simulation path (lbib_set_populations + lbib_read_ib_force).

Callers that cannot allocate device memory -- host callbacks, allocator-
owning host applications, loops that must not allocate after start-up --
use this call with their own device buffers; its only scratch is a static
device array shared by every call.  Two calls in a row with different
particles and populations must each match the simulation path, so nothing
left in the shared scratch by the first call can leak into the second.
This file is named to run last in the suite."""
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


def case(O, seed, shape, xc, yc, theta, walls):
    rng = np.random.default_rng(seed)
    nx, ny = 90, 48
    cfg = dict(nx=nx, ny=ny, wall_bottom=walls, wall_top=walls, tau=0.9,
               u_top=0.0 if walls == "periodic" else 0.02)
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


def test_noalloc_ib_force_matches_simulation_path_twice(O):
    torch = pytest.importorskip("torch")
    from paper_1808_01448_gb300 import build, lbib
    build.build()
    _, _, w, _ = O.lattice()
    cases = [case(O, 21, "ar2", 44.3, 17.6, 0.4, "bounce_back"),
             case(O, 22, "circle", 20.7, 9.2, 0.0, "zou_he")]
    for cfg, f, part in cases:
        ny, nx = cfg["ny"], cfg["nx"]
        dev = torch.tensor((f - w[:, None, None]).astype(np.float32), device="cuda")
        fx = torch.full((ny, nx), np.nan, dtype=torch.float64, device="cuda")
        fy = torch.full((ny, nx), np.nan, dtype=torch.float64, device="cuda")
        lbib.ib_force_noalloc(cfg, dev.data_ptr(), part["vx"], part["vy"], part["xc"],
                              part["yc"], part["theta"], fx_dev_ptr=fx.data_ptr(),
                              fy_dev_ptr=fy.data_ptr())
        torch.cuda.synchronize()
        gx, gy = fx.cpu().numpy(), fy.cpu().numpy()
        rx, ry = reference(lbib, cfg, f, part)
        scale = max(np.abs(rx).max(), np.abs(ry).max())
        assert scale > 1e-5
        np.testing.assert_allclose(gx, rx, rtol=0, atol=1e-6 * scale)
        np.testing.assert_allclose(gy, ry, rtol=0, atol=1e-6 * scale)


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
