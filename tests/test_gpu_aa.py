"""In-place (AA-pattern) streaming against A/B streaming.

With stream_mode "aa" a simulation keeps one population buffer instead of
two; the steps alternate between reading a node's own slots and writing its
neighbours' and the reverse.  Every value goes through the same operations
as in the A/B pull (including the moving-wall term of bounce-back), so the
results are the same bits: populations, fields, particle states and bonds,
after odd and even step counts, alone or in a batch with A/B members,
through a checkpoint, in every storage format and wall kind."""
import numpy as np
import pytest

from paper_1808_01448_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1808_01448_gb300 import build, lbib
    build.build()
    return lbib


def case(walls, storage, nx=96, ny=40, shape="ar2", sim_id=3):
    cfg = W.shear_channel(nx, ny, 1.0, tau=0.9, k_f=0.85, k_r0=0.03, kBT=0.02, seed=5,
                          sim_id=sim_id, hamaker=1e-6)
    cfg["y_cr"] = 1.0
    cfg["wall_bottom"] = cfg["wall_top"] = walls
    if walls == "bounce_back":
        cfg["u_bottom"] = -0.3 * cfg["u_top"]       # both walls moving
    if walls == "periodic":
        cfg.update(u_top=0.0, gx=2e-6, gy=-5e-7)
    p = W.adhesion_particle(cfg, shape, 6.0, x=nx / 3, ligand_density=0.7, sigma=0.02,
                            gap_over_h=0.3 / (ny - 1))
    if walls == "periodic":
        p["yc"] = ny / 2.0
    return cfg, p


def make(L, cfg, p, storage, mode):
    s = L.Sim(storage=storage, stream_mode=mode, **cfg)
    s.add_particle(**p)
    return s


def same(a, b):
    np.testing.assert_array_equal(a.populations(), b.populations())
    for fa, fb in zip(a.fields(), b.fields()):
        np.testing.assert_array_equal(fa, fb)
    assert a.particle(0) == b.particle(0)
    np.testing.assert_array_equal(a.bonds(0)[0], b.bonds(0)[0])
    np.testing.assert_array_equal(a.bonds(0)[1], b.bonds(0)[1])


@pytest.mark.parametrize("walls", ["bounce_back", "zou_he", "periodic"])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "f64"])
def test_in_place_equals_ab(L, walls, storage):
    cfg, p = case(walls, storage)
    ab = make(L, cfg, p, storage, "ab")
    aa = make(L, cfg, p, storage, "aa")
    for n in (37, 27):            # odd, then even in all
        ab.step(n)
        aa.step(n)
        same(ab, aa)
    assert sum(int(ab.bonds(0)[0].sum()) for _ in [0]) >= 0
    ab.close()
    aa.close()


def test_in_place_batch_with_ab_members_and_memory(L):
    cfgs = [case("zou_he", "f32", nx=128, ny=48, shape="circle", sim_id=k) for k in range(2)]
    cfgs.append(case("bounce_back", "f32", nx=100, ny=44, sim_id=5))
    solo = [make(L, c, p, "f32", "ab") for c, p in cfgs]
    mixed = [make(L, c, p, "f32", mode) for (c, p), mode in zip(cfgs, ("aa", "ab", "aa"))]
    for s in solo:
        s.step(71)
    b = L.Batch(mixed)
    assert b.autotune(3)[0] >= 0          # nothing to time with an in-place member
    b.step(40)
    b.step(31)
    b.synchronize()
    for a, c in zip(solo, mixed):
        same(a, c)
    # half the population memory
    n = cfgs[0][0]["nx"] * cfgs[0][0]["ny"]
    assert solo[0].device_bytes() - mixed[0].device_bytes() >= 9 * n * 4
    b.close()
    for s in solo + mixed:
        s.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_in_place_checkpoint_and_populations(L, O, storage):
    cfg, p = case("bounce_back", storage)
    a = make(L, cfg, p, storage, "aa")
    a.step(33)                     # odd: the buffer holds the pushed layout
    blob = a.checkpoint()
    a.step(20)
    b = make(L, cfg, p, storage, "aa")
    b.restore(blob)
    b.step(20)
    same(a, b)
    # a checkpoint of one streaming mode does not load into the other
    c = make(L, cfg, p, storage, "ab")
    with pytest.raises(L.LbibError):
        c.restore(blob)
    # initial populations given from the host, then stepped: as A/B
    rng = np.random.default_rng(4)
    f0 = np.empty((9, cfg["ny"], cfg["nx"]))
    rho = 1 + W.smooth_field(rng, cfg["nx"], cfg["ny"], 0.01)
    ux, uy = (W.smooth_field(rng, cfg["nx"], cfg["ny"], 0.01) for _ in range(2))
    for y in range(cfg["ny"]):
        for x in range(cfg["nx"]):
            f0[:, y, x] = O.equilibrium(rho[y, x], ux[y, x], uy[y, x])
    d = make(L, cfg, p, storage, "aa")
    e = make(L, cfg, p, storage, "ab")
    for s in (d, e):
        s.set_populations(f0)
        s.step(15)
    same(d, e)
    for s in (a, b, c, d, e):
        s.close()
