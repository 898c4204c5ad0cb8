"""GPU path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 storage runs the same arithmetic in double, so fields and
trajectories agree to rounding (1e-11 relative) and bond states bit for bit.
FP32 storage keeps f - w_i in single precision with FP32 collision: velocity
within 1e-5 relative L2 and particle trajectories within 1e-4 lattice units.
"""
import numpy as np
import pytest

from _parity import bonds_every_step
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


def pair(O, L, cfg, particles=(), storage="f64", f_post=None):
    o = O.OracleSim(**cfg)
    g = L.Sim(storage=storage, **cfg)
    for p in particles:
        o.add_particle(**p)
        g.add_particle(**p)
    if f_post is not None:
        o.set_populations(f_post)
        g.set_populations(f_post)
    return o, g


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


WALLS = [("bounce_back", dict(u_top=0.01, gx=2e-6)), ("zou_he", dict(u_top=0.01)),
         ("periodic", dict(gx=1e-6, gy=-5e-7))]


def random_start(O, nx, ny, seed, amp=0.01):
    rng = np.random.default_rng(seed)
    rho = 1 + W.smooth_field(rng, nx, ny, 0.01)
    return eq_field(O, rho, W.smooth_field(rng, nx, ny, amp), W.smooth_field(rng, nx, ny, amp))


@pytest.mark.parametrize("walls,extra", WALLS)
def test_lattice_parity_f64(O, L, walls, extra):
    nx, ny = 37, 23    # ragged: not a multiple of the 256-node tile
    cfg = dict(nx=nx, ny=ny, wall_bottom=walls, wall_top=walls, tau=0.7, **extra)
    f0 = random_start(O, nx, ny, 1)
    o, g = pair(O, L, cfg, f_post=f0)
    for n in (1, 4, 33):
        o.step(n)
        g.step(n)
        np.testing.assert_allclose(g.populations(), o.populations(), rtol=0, atol=1e-13)
    for a, b in zip(g.fields(), o.fields()):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)
    assert g.step_count == o.step_count == 38


@pytest.mark.parametrize("walls,extra", WALLS)
def test_lattice_parity_f32(O, L, walls, extra):
    nx, ny = 300, 41
    cfg = dict(nx=nx, ny=ny, wall_bottom=walls, wall_top=walls, tau=0.8, **extra)
    f0 = random_start(O, nx, ny, 2, amp=1e-3)
    o, g = pair(O, L, cfg, storage="f32", f_post=f0)
    o.step(70)
    g.step(70)
    ro, uo, vo = o.fields()
    rg, ug, vg = g.fields()
    assert rel_l2(np.stack([ug, vg]), np.stack([uo, vo])) < 1e-5
    np.testing.assert_allclose(rg, ro, rtol=0, atol=1e-7)


@pytest.mark.parametrize("walls", ["bounce_back", "zou_he", "periodic"])
@pytest.mark.parametrize("shape", ["circle", "ar3"])
def test_ib_force_parity(O, L, walls, shape):
    nx, ny = 80, 44
    cfg = dict(nx=nx, ny=ny, wall_bottom=walls, wall_top=walls, tau=0.9,
               u_top=0.0 if walls == "periodic" else 0.02)
    f0 = random_start(O, nx, ny, 3, amp=0.01)
    vx, vy = W.particle_outline(shape, 7.0)
    p = dict(vx=vx, vy=vy, xc=41.3, yc=12.6 if walls != "periodic" else 2.2, theta=0.3,
             ligand_density=0.0, sigma=0.0)
    o, g = pair(O, L, cfg, [p], f_post=f0)
    fo = o.ib_force()
    fg = g.ib_force()
    scale = max(np.abs(fo[0]).max(), np.abs(fo[1]).max())
    assert scale > 1e-4
    np.testing.assert_allclose(fg[0], fo[0], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(fg[1], fo[1], rtol=0, atol=1e-12 * scale)
    assert abs(fg[0].sum() - fo[0].sum()) < 1e-12 * scale * nx


def adhesion_case(shape="ar2", Re=1.0, nx=96, ny=40, rl=0.7, sigma=0.02, seed=5, r=6.0):
    """Particle released 0.3 lu above the bottom Zou-He wall of a shear
    channel, with soft bonds (y_cr = 1, sigma = 0.02) so that bonds form and
    the weakly coupled step stays stable for a small, light particle."""
    cfg = W.shear_channel(nx, ny, Re, tau=0.9, k_f=0.85, k_r0=1e-3, kBT=0.02, seed=seed,
                          sim_id=2, hamaker=1e-6)
    cfg["y_cr"] = 1.0
    p = W.adhesion_particle(cfg, shape, r, x=nx / 3, ligand_density=rl, sigma=sigma,
                            gap_over_h=0.3 / (ny - 1))
    return cfg, p


def test_full_step_parity_f64_with_bonds(O, L):
    """Whole coupled step in FP64 storage: trajectories agree to rounding and
    bond states bit for bit at every step."""
    cfg, p = adhesion_case()
    o, g = pair(O, L, cfg, [p])
    total_bonded = 0
    for t in range(120):
        o.step(1)
        g.step(1)
        bo, ao = o.bonds(0)
        bg, ag = g.bonds(0)
        assert np.array_equal(bo, bg), f"bond states differ at step {t + 1}"
        np.testing.assert_allclose(ag[bg == 1], ao[bo == 1], rtol=0, atol=1e-9)
        total_bonded += int(bg.sum())
        # the step's loads, side by side: wall force (Eq. 12), hydrodynamic
        # and bond moments (Eq. 7-9)
        po, pg = o.particle(0), g.particle(0)
        assert po["Fw"][1] != 0.0
        assert pg["Fw"][0] == po["Fw"][0] == 0.0
        assert pg["Fw"][1] == pytest.approx(po["Fw"][1], rel=1e-9), f"Fw at step {t + 1}"
        assert pg["Mb"] == pytest.approx(po["Mb"], rel=1e-9, abs=1e-15), f"Mb at step {t + 1}"
        np.testing.assert_allclose(pg["Fb"], po["Fb"], rtol=1e-9, atol=1e-15)
        assert pg["Mh"] == pytest.approx(po["Mh"], rel=1e-6, abs=1e-12), f"Mh at step {t + 1}"
        for k in ("gap_bottom", "gap_top"):
            assert pg[k] == pytest.approx(po[k], abs=1e-12), f"{k} at step {t + 1}"
    assert total_bonded > 0          # the case exercises bond formation
    po, pg = o.particle(0), g.particle(0)
    for k in ("xc", "yc", "theta", "u", "v", "omega"):
        assert pg[k] == pytest.approx(po[k], abs=1e-10), k
    for k in ("Fh", "Fb"):
        np.testing.assert_allclose(pg[k], po[k], rtol=1e-7, atol=1e-13)
    assert pg["n_probing"] == po["n_probing"] and pg["n_bonded"] == po["n_bonded"]
    ro, uo, vo = o.fields()
    rg, ug, vg = g.fields()
    assert rel_l2(np.stack([ug, vg]), np.stack([uo, vo])) < 1e-11


def test_moving_near_box_parity_f64(O, L):
    """A particle carried across the lattice's work tiles and around the
    periodic y boundary (a fully periodic box whose fluid the body force
    accelerates in y): the bulk pass skips the near box through per-tile
    counts that the near-box pass moves with the box every step, so a count
    left behind would let the bulk pass overwrite a near-box node.  FP64
    storage against the oracle to rounding after 400 steps, the particle
    having risen across more than one tile's rows."""
    nx, ny = 96, 64
    cfg = dict(nx=nx, ny=ny, wall_bottom="periodic", wall_top="periodic", tau=0.8, gy=2e-4,
               hamaker=0.0, seed=3, sim_id=0)
    vx, vy = W.circle_polygon(6.0, 40)
    p = dict(vx=vx, vy=vy, xc=40.0, yc=ny - 14.0, theta=0.0, rho_p=1.0, ligand_density=0.0,
             sigma=0.02)
    o, g = pair(O, L, cfg, [p])
    y0 = g.particle(0)["yc"]
    o.step(400)
    g.step(400)
    po, pg = o.particle(0), g.particle(0)
    rise = pg["yc"] - y0
    assert rise > 1024 / nx + 1, f"the particle rose only {rise:.2f} rows"
    for k in ("xc", "yc", "theta", "u", "v", "omega"):
        assert pg[k] == pytest.approx(po[k], abs=1e-10), k
    ro, uo, vo = o.fields()
    rg, ug, vg = g.fields()
    assert rel_l2(np.stack([ug, vg]), np.stack([uo, vo])) < 1e-11


def test_set_populations_from_page_locked_memory(O, L):
    """The import reads page-locked host memory in place and any other host
    memory through a device copy: the same state either way, before and
    after stepping."""
    import torch
    cfg = dict(nx=64, ny=32, wall_bottom="bounce_back", wall_top="bounce_back", tau=0.8,
               u_top=0.01, seed=2, sim_id=0)
    f = random_start(O, 64, 32, 7)
    pinned = torch.from_numpy(f.copy()).pin_memory()
    a = L.Sim(storage="f32", **cfg)
    b = L.Sim(storage="f32", **cfg)
    a.set_populations(f)
    b.set_populations(pinned.numpy())
    np.testing.assert_array_equal(a.populations(), b.populations())
    a.step(10)
    b.step(10)
    np.testing.assert_array_equal(a.populations(), b.populations())
    a.close()
    b.close()


def test_catch_bond_parity_f64(O, L):
    """Catch bonds (sigma* = 2 sigma in Eq. 11: a stretched bond breaks less
    often): bond states bit for bit with the oracle at every step, and the
    adhesion probability n_bonded / n_probing of the oracle's counts."""
    cfg, p = adhesion_case()
    cfg["sigma_star_ratio"] = 2.0
    o, g = pair(O, L, cfg, [p])
    for t in range(100):
        o.step(1)
        g.step(1)
        assert np.array_equal(o.bonds(0)[0], g.bonds(0)[0]), f"step {t + 1}"
    po, pg = o.particle(0), g.particle(0)
    assert pg["n_bonded"] > 0
    assert pg["p_adhesion"] == po["n_bonded"] / po["n_probing"]
    assert pg["xc"] == pytest.approx(po["xc"], abs=1e-10)


def test_critical_length_sweep(L):
    """The paper's Fig. 7 study: a longer critical bond length lets more
    ligands probe the wall and more bonds form."""
    sims = []
    for cfg, parts in W.ycr_sweep():
        s = L.Sim(storage="f32", **cfg)
        for q in parts:
            s.add_particle(**q)
        sims.append(s)
    b = L.Batch(sims)
    probing, bonded = [0] * len(sims), [0] * len(sims)
    for _ in range(20):
        b.step(100)
        for i, s in enumerate(sims):
            st = s.particle(0)
            probing[i] += st["n_probing"]
            bonded[i] += st["n_bonded"]
    assert probing[0] < probing[1] < probing[2]
    assert bonded[0] < bonded[2]
    b.close()


@pytest.mark.parametrize("shape", ["circle", "ar3"])
def test_full_step_parity_f32(O, L, shape):
    """FP32 storage against the oracle for 200 coupled steps: bond flags at
    every step (a difference only at a logged near tie), then velocity and
    trajectory within the FP32 tolerances."""
    cfg, p = adhesion_case(shape=shape, Re=0.1, nx=128, ny=48, r=7.0)
    o, g = pair(O, L, cfg, [p], storage="f32")
    bonds_every_step([(o, g)], lambda: g.step(1), 200, f"f32 {shape}")
    ro, uo, vo = o.fields()
    rg, ug, vg = g.fields()
    assert rel_l2(np.stack([ug, vg]), np.stack([uo, vo])) < 1e-5
    po, pg = o.particle(0), g.particle(0)
    for k in ("xc", "yc", "theta"):
        assert abs(pg[k] - po[k]) < 1e-4, k


def test_step_without_overlap_when_near_box_exceeds_lattice(O, L):
    """A particle whose near box (force tile + 8) is wider than the lattice
    is stepped with the plain lattice pass instead of the overlapped
    bulk/near split; results still follow the oracle."""
    cfg, p = adhesion_case(nx=30, ny=40, r=8.0, shape="circle")
    p["xc"] = 15.0
    o, g = pair(O, L, cfg, [p])
    o.step(40)
    g.step(40)
    po, pg = o.particle(0), g.particle(0)
    for k in ("xc", "yc", "theta"):
        assert pg[k] == pytest.approx(po[k], abs=1e-10), k
    ro, uo, vo = o.fields()
    rg, ug, vg = g.fields()
    assert rel_l2(np.stack([ug, vg]), np.stack([uo, vo])) < 1e-11


def test_poiseuille_circle_workload_f32(O, L):
    """Single circle of radius 10 (63 markers) in the 200 x 50 body-force
    channel with bounce-back walls, tau 0.8, Re 0.1."""
    cfg, parts = W.poiseuille_circle()
    o, g = pair(O, L, cfg, parts, storage="f32")
    o.step(150)
    g.step(150)
    ro, uo, vo = o.fields()
    rg, ug, vg = g.fields()
    assert rel_l2(np.stack([ug, vg]), np.stack([uo, vo])) < 1e-5
    po, pg = o.particle(0), g.particle(0)
    for k in ("xc", "yc", "theta"):
        assert abs(pg[k] - po[k]) < 1e-4


def test_full_size_workload_sampled(O, L):
    """1024 x 256 channel with an equal-area ellipse of aspect ratio 3 at
    Re = 1 in FP32, as the benchmark runs it (batched with a second sim):
    fields and trajectory after 12 steps match the oracle."""
    sims = W.single_ellipse_sweep(shapes=("ar3",), reynolds=(1.0, 0.1))
    gs, os_ = [], []
    for cfg, parts in sims:
        o, g = pair(O, L, cfg, parts, storage="f32")
        gs.append(g)
        os_.append(o)
    b = L.Batch(gs)
    b.step(12)
    for o, g in zip(os_, gs):
        o.step(12)
        ro, uo, vo = o.fields()
        rg, ug, vg = g.fields()
        assert rel_l2(np.stack([ug, vg]), np.stack([uo, vo])) < 1e-5
        po, pg = o.particle(0), g.particle(0)
        assert abs(pg["xc"] - po["xc"]) < 1e-6 and abs(pg["yc"] - po["yc"]) < 1e-6
    b.close()


def test_batch_equals_solo(L):
    """Stepping in a batch (uneven lattices, graph replays and a ragged
    remainder) gives bit-identical results to stepping alone."""
    specs = [(64, 32, "circle"), (200, 50, "ar2"), (150, 40, "ar3")]

    def make(i, nx, ny, shape):
        cfg, p = adhesion_case(shape=shape, nx=nx, ny=ny, seed=9)
        cfg["sim_id"] = i
        s = L.Sim(storage="f32", **cfg)
        s.add_particle(**p)
        return s

    solo = [make(i, *sp) for i, sp in enumerate(specs)]
    mixed = [make(i, *sp) for i, sp in enumerate(specs)]
    for s in solo:
        s.step(71)
    b = L.Batch(mixed)
    b.step(40)
    b.step(31)
    for a, c in zip(solo, mixed):
        np.testing.assert_array_equal(a.populations(), c.populations())
        pa, pc = a.particle(0), c.particle(0)
        assert pa == pc
        np.testing.assert_array_equal(a.bonds(0)[0], c.bonds(0)[0])
    b.close()


def test_edge_cases(O, L):
    s = L.Sim(nx=8, ny=4, tau=0.7, wall_bottom="periodic", wall_top="periodic")
    s.step(0)
    assert s.step_count == 0
    with pytest.raises(L.LbibError) as e:
        s.step(-1)
    assert e.value.status == "E_ARG"
    s.step(65)
    f = s.populations()
    np.testing.assert_allclose(f.sum(axis=0), 1.0, atol=1e-6)
    g = L.Sim(nx=64, ny=32)
    with pytest.raises(L.LbibError):
        g.add_particle(*W.circle_polygon(40.0, 200), xc=30, yc=16)   # tile wider than lattice
    with pytest.raises(L.LbibError):
        g.set_receptors(2, 1.0)
    g.add_particle(*W.circle_polygon(4.0, 25), xc=30, yc=16)
    g.step(3)
    with pytest.raises(L.LbibError) as e:
        g.add_particle(*W.circle_polygon(4.0, 25), xc=10, yc=16)
    assert e.value.status == "E_STATE"
    with pytest.raises(L.LbibError) as e:
        g.set_populations(np.ones((9, 32, 64)))
    assert e.value.status == "E_STATE"


def test_instability_is_reported(L):
    # a body force far beyond the lattice's range drives the state non-finite
    s = L.Sim(nx=32, ny=16, wall_bottom="periodic", wall_top="periodic", tau=0.51, gx=0.2)
    s.step(300)
    with pytest.raises(L.LbibError) as e:
        s.synchronize()
    assert e.value.status == "E_UNSTABLE"


def test_generated_outline_matches_explicit_polygon(L):
    """lbib_add_particle with shape parameters builds the same ellipse as the
    explicit equal-arc-length polygon (to the arc-length table's accuracy)."""
    s = L.Sim(nx=128, ny=64)
    s.add_particle(shape=1, a=6.0, b=12.0, xc=64, yc=32, ligand_density=0.5)
    vx, vy = W.ellipse_polygon(6.0, 12.0, W.n_markers(6.0, 12.0))
    t = L.Sim(nx=128, ny=64)
    t.add_particle(vx, vy, xc=64, yc=32, ligand_density=0.5)
    a, b = s.particle(0), t.particle(0)
    assert a["nl"] == b["nl"]
    assert a["area"] == pytest.approx(b["area"], rel=1e-6)
    assert a["inertia"] == pytest.approx(b["inertia"], rel=1e-5)


def test_kernel_timing(L):
    cfg, p = adhesion_case(nx=256, ny=64)
    s = L.Sim(storage="f32", **cfg)
    s.add_particle(**p)
    b = L.Batch([s])
    b.set_timing(4)
    b.step(32 * 16)
    t = b.kernel_times()
    assert t["lattice_n"] == 4 and t["particle_n"] == 4 and t["near_n"] == 4
    assert 0 < t["lattice_ms"] < 5 and 0 < t["particle_ms"] < 5 and 0 < t["near_ms"] < 5
    b.close()


def test_torch_allocator_and_stream(O, L):
    torch = pytest.importorskip("torch")
    st = torch.cuda.Stream()
    alloc = L.torch_allocator()
    cfg, p = adhesion_case(nx=64, ny=32)
    before = torch.cuda.memory_allocated()
    g = L.Sim(storage="f64", stream=st.cuda_stream, allocator=alloc, **cfg)
    g.add_particle(**p)
    assert torch.cuda.memory_allocated() > before
    o = O.OracleSim(**cfg)
    o.add_particle(**p)
    g.step(40)
    o.step(40)
    assert abs(g.particle(0)["xc"] - o.particle(0)["xc"]) < 1e-11
    g.close()


@pytest.mark.parametrize("walls", ["zou_he", "periodic"])
def test_multi_direct_forcing_parity_f64(O, L, walls):
    """Three direct-forcing passes (multi-direct forcing): the IB force field
    of the GPU's FP64 path equals the oracle's to rounding."""
    nx, ny = 80, 44
    cfg = dict(nx=nx, ny=ny, wall_bottom=walls, wall_top=walls, tau=0.9,
               u_top=0.0 if walls == "periodic" else 0.02, ib_iterations=3)
    f0 = random_start(O, nx, ny, 4, amp=0.01)
    vx, vy = W.particle_outline("ar2", 7.0)
    p = dict(vx=vx, vy=vy, xc=40.6, yc=14.3 if walls != "periodic" else 2.2, theta=0.2,
             ligand_density=0.0, sigma=0.0)
    o, g = pair(O, L, cfg, [p], f_post=f0)
    fo = o.ib_force()
    fg = g.ib_force()
    scale = max(np.abs(fo[0]).max(), np.abs(fo[1]).max())
    assert scale > 1e-4
    np.testing.assert_allclose(fg[0], fo[0], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(fg[1], fo[1], rtol=0, atol=1e-12 * scale)
    # the passes change the force (against a single pass)
    o1, g1 = pair(O, L, dict(cfg, ib_iterations=1), [p], f_post=f0)
    assert np.abs(g1.ib_force()[0] - fg[0]).max() > 1e-3 * scale


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_multi_direct_forcing_full_step(O, L, storage):
    """Coupled steps with three direct-forcing passes against the oracle:
    FP64 to rounding with bond states equal at every step; FP32 within the
    stated tolerances (velocity 1e-5 relative L2, trajectory 1e-4)."""
    cfg, p = adhesion_case(shape="circle", Re=0.1, nx=112, ny=44, r=6.5)
    cfg["ib_iterations"] = 3
    o, g = pair(O, L, cfg, [p], storage=storage)
    steps = 60 if storage == "f64" else 150
    for t in range(steps):
        o.step(1)
        g.step(1)
        if storage == "f64":
            assert np.array_equal(o.bonds(0)[0], g.bonds(0)[0]), f"step {t + 1}"
    ro, uo, vo = o.fields()
    rg, ug, vg = g.fields()
    err = rel_l2(np.stack([ug, vg]), np.stack([uo, vo]))
    po, pg = o.particle(0), g.particle(0)
    if storage == "f64":
        assert err < 1e-11
        for k in ("xc", "yc", "theta", "u", "v", "omega"):
            assert pg[k] == pytest.approx(po[k], abs=1e-10), k
    else:
        assert err < 1e-5
        for k in ("xc", "yc", "theta"):
            assert abs(pg[k] - po[k]) < 1e-4, k
        assert np.array_equal(o.bonds(0)[0], g.bonds(0)[0])


def test_ib_iterations_out_of_range_is_refused(L):
    with pytest.raises(L.LbibError):
        L.Sim(nx=32, ny=16, ib_iterations=17)
