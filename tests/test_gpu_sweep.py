"""The batched design sweep on the GPU: 72 uneven channels (shape x ligand
density x bond strength x Re, lattices 256..1024 x 64..256) stepped in one
batch.  Members give the same bits as when stepped alone, and the smallest
member follows the FP64 oracle within the FP32 tolerances (velocity 1e-5
relative L2, trajectory 1e-4 lattice units, bond states equal).
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


def make(L, cfg, parts, storage="f32"):
    s = L.Sim(storage=storage, **cfg)
    for p in parts:
        s.add_particle(**p)
    return s


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_design_sweep_batch_equals_solo(L):
    sweep = W.design_sweep()
    assert len(sweep) == 72
    sims = [make(L, c, p) for c, p in sweep]
    b = L.Batch(sims)
    b.step(32)          # one captured graph
    b.step(9)           # ragged remainder, odd parity
    sizes = [c["nx"] * c["ny"] for c, _ in sweep]
    picks = sorted({0, 35, 71, int(np.argmin(sizes)), int(np.argmax(sizes))})
    for i in picks:
        c, p = sweep[i]
        solo = make(L, c, p)
        solo.step(41)
        np.testing.assert_array_equal(solo.populations(), sims[i].populations())
        assert solo.particle(0) == sims[i].particle(0)
        np.testing.assert_array_equal(solo.bonds(0)[0], sims[i].bonds(0)[0])
        solo.close()
    b.close()
    for s in sims:
        s.close()


def test_design_sweep_smallest_member_vs_oracle(O, L):
    sweep = W.design_sweep()
    sizes = [c["nx"] * c["ny"] for c, _ in sweep]
    order = np.argsort(sizes, kind="stable")
    sims = [make(L, c, p) for c, p in sweep]
    b = L.Batch(sims)
    oracles = {}
    for i in order[:2]:
        c, p = sweep[int(i)]
        o = O.OracleSim(**c)
        for q in p:
            o.add_particle(**q)
        oracles[int(i)] = o
    # bond flags of both members against their oracles at every step of the
    # batched stepping
    bonds_every_step([(oracles[i], sims[i]) for i in oracles], lambda: b.step(1), 64,
                     "sweep member")
    for i in order[:2]:
        o = oracles[int(i)]
        ro, uo, vo = o.fields()
        rg, ug, vg = sims[int(i)].fields()
        assert rel_l2(np.stack([ug, vg]), np.stack([uo, vo])) < 1e-5
        po, pg = o.particle(0), sims[int(i)].particle(0)
        for k in ("xc", "yc", "theta"):
            assert abs(pg[k] - po[k]) < 1e-4, k
    b.close()
    for s in sims:
        s.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_lattice_variants_give_identical_bits(L, storage):
    """Every lattice-pass kernel variant computes the same bits, and tuning
    (timing runs of each variant) leaves the simulations unchanged."""
    sweep = W.design_sweep()[:5]
    runs = []
    for v in range(L.LATTICE_VARIANTS):
        sims = [make(L, c, p, storage) for c, p in sweep]
        b = L.Batch(sims)
        b.step(3)
        if v == 0:
            before = [s.populations() for s in sims]
            steps = [s.step_count for s in sims]
            best, ms = b.autotune(3)
            assert 0 <= best < L.LATTICE_VARIANTS and all(m > 0 for m in ms)
            for s, f, n in zip(sims, before, steps):
                np.testing.assert_array_equal(s.populations(), f)
                assert s.step_count == n
        b.set_variant(v)
        b.step(37)
        runs.append([(s.populations(), s.particle(0)) for s in sims])
        b.close()
        for s in sims:
            s.close()
    for other in runs[1:]:
        for (fa, pa), (fb, pb) in zip(runs[0], other):
            np.testing.assert_array_equal(fa, fb)
            assert pa == pb


@pytest.mark.parametrize("clean", [False, True])
def test_flushed_steps_equal_plain_steps(L, clean):
    """Stepping with an L2 flush before every step (the cold-L2 timing form)
    gives the same bits as plain stepping, over a full graph and an odd
    remainder, and reports positive step, bulk-pass and flush times."""
    import torch
    sweep = W.design_sweep()[:4]
    plain = [make(L, c, p) for c, p in sweep]
    flushed = [make(L, c, p) for c, p in sweep]
    bp, bf = L.Batch(plain), L.Batch(flushed)
    bp.step(37)
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    buf = torch.empty(2 * l2 + 4096, dtype=torch.uint8, device="cuda")
    t = bf.step_flushed(37, buf.data_ptr(), buf.numel(), clean)
    assert t["step_ms"] > 0 and t["bulk_ms"] > 0 and t["flush_ms"] > 0
    assert t["bulk_ms"] <= t["step_ms"]
    for a, b in zip(plain, flushed):
        assert a.step_count == b.step_count == 37
        np.testing.assert_array_equal(a.populations(), b.populations())
        assert a.particle(0) == b.particle(0)
    with pytest.raises(L.LbibError):
        bf.step_flushed(1, buf.data_ptr(), 1 << 20, clean)     # smaller than L2
    bf.step(5)
    bp.step(5)
    for a, b in zip(plain, flushed):
        np.testing.assert_array_equal(a.populations(), b.populations())
    bp.close()
    bf.close()
    for s in plain + flushed:
        s.close()


def test_batch_readback_equals_per_sim_readback(L):
    """One batched readback of every member's particle states gives exactly
    what each simulation's own readback gives, and counts its bytes."""
    sweep = W.design_sweep()[:7]
    sims = [make(L, c, p) for c, p in sweep]
    b = L.Batch(sims)
    b.step(35)
    rows = b.particles()
    assert len(rows) == len(sims)
    for s, row in zip(sims, rows):
        assert row == s.particles()
    assert b.last_d2h_bytes > 0
    b.close()
    for s in sims:
        s.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_particle_cta_widths_give_identical_bits(L, storage):
    """256- and 512-thread particle CTAs compute the same bits (over a full
    graph and an odd remainder); widths that do not fit are refused."""
    sweep = W.design_sweep()[:6]
    runs = []
    for width in (512, 256):
        sims = [make(L, c, p, storage) for c, p in sweep]
        b = L.Batch(sims)
        b.set_particle_threads(width)
        b.step(37)
        runs.append([(s.populations(), s.particles(), s.bonds(0)[0]) for s in sims])
        with pytest.raises(L.LbibError):
            b.set_particle_threads(384)
        b.close()
        for s in sims:
            s.close()
    for (fa, pa, ba), (fb, pb, bb) in zip(*runs):
        np.testing.assert_array_equal(fa, fb)
        assert pa == pb
        np.testing.assert_array_equal(ba, bb)


def test_async_readback_gives_the_states_when_started(L):
    """A readback started after 35 steps and collected after 10 more gives
    the states after 35 steps; a second start before collection is refused."""
    sweep = W.design_sweep()[:5]
    a = [make(L, c, p) for c, p in sweep]
    b = [make(L, c, p) for c, p in sweep]
    ba, bb = L.Batch(a), L.Batch(b)
    ba.step(35)
    ba.read_particles_async()
    with pytest.raises(L.LbibError):
        ba.read_particles_async()
    ba.step(10)
    late = ba.particles()
    bb.step(35)
    assert late == bb.particles()
    bb.step(10)
    assert ba.particles() == bb.particles()
    ba.close()
    bb.close()
    for s in a + b:
        s.close()


def test_batch_synchronize_reports_a_member_error(L):
    """A batch's synchronize (one copy of the members' error words) reports
    an unstable member and stays quiet for a stable batch, and it leaves a
    started readback pending."""
    sweep = W.design_sweep()[:3]
    good = [make(L, c, p) for c, p in sweep]
    b = L.Batch(good)
    b.step(5)
    b.read_particles_async()
    b.step(5)
    b.synchronize()
    at5 = b.particles()             # the readback started after 5 steps
    at10 = b.particles()
    assert len(at5) == len(at10) == 3 and at5 != at10
    b.close()
    bad = L.Sim(nx=32, ny=16, wall_bottom="periodic", wall_top="periodic", tau=0.51, gx=0.2)
    mixed = L.Batch([good[0], bad])
    mixed.step(300)
    with pytest.raises(L.LbibError) as e:
        mixed.synchronize()
    assert e.value.status == "E_UNSTABLE"
    mixed.close()
    for s in good + [bad]:
        s.close()


def test_member_reads_wait_for_the_batch(L):
    """A member's own read calls see every step its batch enqueued, although
    the batch steps on another stream (the first member's): populations and
    bonds read right after stepping equal those read after synchronising
    the batch."""
    sweep = W.design_sweep()[:4]
    sims = [make(L, c, p) for c, p in sweep]
    b = L.Batch(sims)
    for _ in range(3):
        b.step(5)
        early = [sims[k].populations() for k in (1, 3)]
        b.synchronize()
        for f, k in zip(early, (1, 3)):
            np.testing.assert_array_equal(f, sims[k].populations())
    b.close()
    for s in sims:
        s.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_graph_chunks_equal_direct_steps(L, storage):
    """A call's steps run as 32-step graphs, then 4-step graphs, then direct
    launches; any split of the same steps gives the same bits: 45 steps in
    one call (32 + 3 x 4 + 1), in calls of 7, and one at a time."""
    sweep = W.design_sweep()[:3]
    results = []
    for split in ([45], [7] * 6 + [3], [1] * 45):
        sims = [make(L, c, p, storage) for c, p in sweep]
        b = L.Batch(sims)
        for n in split:
            b.step(n)
        b.synchronize()
        results.append([(s.populations(), s.particle(0), s.step_count) for s in sims])
        b.close()
        for s in sims:
            s.close()
    for other in results[1:]:
        for (fa, pa, na), (fb, pb, nb) in zip(results[0], other):
            np.testing.assert_array_equal(fa, fb)
            assert pa == pb and na == nb == 45
