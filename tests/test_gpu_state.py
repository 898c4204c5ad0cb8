"""Simulation state from the host: checkpoints (bit-identical resume),
particle records, device-memory accounting, and failure detection without a
GPU fault -- an allocator that fails on its n-th call (LBIB_E_OOM, handles
still destroyable) and a bounded device wait that runs out (LBIB_E_TIMEOUT,
the context still usable)."""
import ctypes as C
import os

import numpy as np
import pytest

from paper_1808_01448_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1808_01448_gb300 import build, lbib
    build.build()
    return lbib


def two_particle_case(storage, sim_id=4):
    cfg = W.shear_channel(160, 48, 1.0, tau=0.9, k_f=0.85, k_r0=0.03, kBT=0.02, seed=8,
                          sim_id=sim_id, hamaker=1e-6)
    cfg["y_cr"] = 1.0
    parts = [W.adhesion_particle(cfg, "ar2", 6.0, x=40.0, ligand_density=0.7, sigma=0.02,
                                 gap_over_h=0.3 / 47),
             W.adhesion_particle(cfg, "circle", 5.0, x=110.0, ligand_density=0.9, sigma=0.02,
                                 gap_over_h=0.5 / 47)]
    return cfg, parts


def make(L, storage, cfg, parts):
    s = L.Sim(storage=storage, **cfg)
    for p in parts:
        s.add_particle(**p)
    return s


@pytest.mark.parametrize("storage,saved_at", [("f32", 51), ("f16", 40), ("f64", 33)])
def test_checkpoint_resume_is_bit_identical(L, storage, saved_at):
    cfg, parts = two_particle_case(storage)
    a = make(L, storage, cfg, parts)
    a.step(saved_at)
    blob = a.checkpoint()
    a.step(70)
    b = make(L, storage, cfg, parts)
    b.restore(blob)
    assert b.step_count == saved_at
    b.step(70)
    assert b.step_count == a.step_count == saved_at + 70
    np.testing.assert_array_equal(a.populations(), b.populations())
    for k in range(2):
        assert a.particle(k) == b.particle(k)
        assert a.record(k) == b.record(k)
        ba, xa = a.bonds(k)
        bb, xb = b.bonds(k)
        np.testing.assert_array_equal(ba, bb)
        np.testing.assert_array_equal(xa, xb)
    assert sum(int(a.bonds(k)[0].sum()) for k in range(2)) > 0
    # a batch steps a restored simulation like any other
    c = make(L, storage, cfg, parts)
    c.restore(blob)
    bt = L.Batch([c])
    bt.step(70)
    bt.synchronize()
    np.testing.assert_array_equal(a.populations(), c.populations())
    bt.close()
    for s in (a, b, c):
        s.close()


def test_checkpoint_rejects_a_mismatched_simulation(L):
    cfg, parts = two_particle_case("f32")
    a = make(L, "f32", cfg, parts)
    a.step(3)
    blob = a.checkpoint()
    other = make(L, "f32", dict(cfg, nx=cfg["nx"] + 32), parts)
    with pytest.raises(L.LbibError) as e:
        other.restore(blob)
    assert e.value.status == "E_ARG"
    one = make(L, "f32", cfg, parts[:1])
    with pytest.raises(L.LbibError):
        one.restore(blob)
    with pytest.raises(L.LbibError):
        a.restore(blob[:100])
    bad = bytearray(blob)
    bad[0:8] = b"NOTACKPT"
    with pytest.raises(L.LbibError):
        a.restore(bytes(bad))
    for s in (a, other, one):
        s.close()


def test_particle_record_roundtrip_and_prescribed_pose(L):
    cfg, parts = two_particle_case("f32")
    s = make(L, "f32", cfg, parts)
    s.step(10)
    r = s.record(1)
    assert r["step"] == 10
    st = s.particle(1)
    assert (r["xc"], r["yc"], r["theta"]) == (st["xc"], st["yc"], st["theta"])
    s.set_record(1, xc=r["xc"] + 3.25, theta=0.4, u=0.0, v=0.0, omega=0.0, xc1=r["xc"] + 3.25,
                 yc1=r["yc"], theta1=0.4, u1=0.0, v1=0.0, omega1=0.0)
    r2 = s.record(1)
    assert r2["xc"] == r["xc"] + 3.25 and r2["theta"] == 0.4 and r2["step"] == 10
    # the IB forcing follows the new pose: the force field's centroid moves
    fx, _ = s.ib_force()
    w = np.abs(fx)
    xs = np.arange(cfg["nx"])
    half = w[:, 80:]
    cx = float((half.sum(axis=0) * xs[80:]).sum() / half.sum())
    assert abs(cx - (r["xc"] + 3.25)) < 1.0
    with pytest.raises(L.LbibError):
        s.set_record(1, xc=float("nan"))
    s.step(5)
    s.synchronize()
    s.close()


def test_device_bytes_accounts_for_populations_and_particles(L):
    cfg, parts = two_particle_case("f32")
    s = make(L, "f32", cfg, parts)
    n = cfg["nx"] * cfg["ny"]
    before = s.device_bytes()
    assert before >= 2 * 9 * n * 4
    s.step(2)
    assert s.device_bytes() >= before
    h = make(L, "f16", cfg, parts)
    assert h.device_bytes() < before
    s.close()
    h.close()


def test_allocator_failure_is_reported_and_handles_stay_destroyable(L):
    """An allocator hook that fails on its n-th call, for every n up to the
    calls a two-particle simulation makes through its first steps and a batch:
    the failing call reports LBIB_E_OOM and every handle made so far is still
    destroyable; afterwards a simulation with a working allocator runs."""
    torch = pytest.importorskip("torch")
    cfg, parts = two_particle_case("f32")
    live = {}

    def run_with(fail_at):
        calls = {"n": 0}

        def _alloc(nbytes, stream, ctx):
            calls["n"] += 1
            if calls["n"] == fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                   stream or 0)
            live[p] = True
            return p

        def _free(ptr, stream, ctx):
            if live.pop(ptr, None):
                torch.cuda.caching_allocator_delete(ptr)

        hook = (L.ALLOC_FN(_alloc), L.FREE_FN(_free))
        made, err = [], None
        try:
            s = L.Sim(storage="f32", allocator=hook, **cfg)
            made.append(s)
            for p in parts:
                s.add_particle(**p)
            s.step(3)
            b = L.Batch([s])
            made.append(b)
            b.step(2)
            s.fields()
        except L.LbibError as e:
            err = e
        for h in reversed(made):
            h.close()
        return calls["n"], err

    total, err = run_with(0)
    assert err is None and total >= 5
    for k in range(1, total + 1):
        _, err = run_with(k)
        assert err is not None and err.status == "E_OOM", k
    assert not live          # everything allocated was given back
    s = make(L, "f32", cfg, parts)
    s.step(4)
    s.synchronize()
    s.close()


@pytest.mark.parametrize("variant", [4, 5])
def test_bounded_wait_reports_timeout(L, monkeypatch, variant):
    """The copy-engine variants of the bulk lattice pass wait for their
    staged copies (and the pipeline's producer for the release of a stage)
    at most LBIB_WAIT_POLLS polls; with 0 polls those waits give up at once
    (each CTA then drains its own copies with a full-length bounded wait
    before it leaves) and the next call reports LBIB_E_TIMEOUT.  The context
    stays usable."""
    cfg, parts = two_particle_case("f32")
    s = make(L, "f32", cfg, parts)
    s.step(2)
    monkeypatch.setenv("LBIB_WAIT_POLLS", "0")
    b = L.Batch([s])
    monkeypatch.delenv("LBIB_WAIT_POLLS")
    b.set_variant(variant)
    b.step(1)
    with pytest.raises(L.LbibError) as e:
        b.synchronize()
    assert e.value.status == "E_TIMEOUT"
    b.close()
    s.close()
    # a fresh batch with the default limit on the same context runs the same
    # variant to completion and matches plain stepping
    t = make(L, "f32", cfg, parts)
    u = make(L, "f32", cfg, parts)
    bt = L.Batch([t])
    bt.set_variant(variant)
    bt.step(6)
    bt.synchronize()
    u.step(6)
    np.testing.assert_array_equal(t.populations(), u.populations())
    bt.close()
    for x in (t, u):
        x.close()
