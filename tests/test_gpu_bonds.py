"""Bond kinetics (Eq. 9-11) of the GPU path against the FP64 oracle, step by
step.

Replay: the GPU particle is given the oracle's pose before every step
(lbib_set_particle_record), so its bond step sees the same geometry.  The
bond geometry, probabilities and anchors are FP64 on every storage path, so
the bond flags equal the oracle's at every step in FP64, FP32, FP16 and BF16
storage, and the anchors agree to FP64 rounding.

Free runs: without replay the FP32 trajectory differs from the oracle's by
up to ~1e-5 lattice units, so a decision whose uniform or gap lies that
close to its threshold may go the other way.  The bond flags are compared at
every step; a difference is allowed only at a step where the oracle logged a
near tie (|U - P| or |gap - y_cr| below the trajectory tolerance 1e-4), and
the first divergence step and the Hamming distance are reported."""
import numpy as np
import pytest

from paper_1808_01448_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NEAR_TIE = 1e-4      # the FP32 trajectory tolerance, lattice units / probability


@pytest.fixture(scope="module")
def L():
    from paper_1808_01448_gb300 import build, lbib
    build.build()
    return lbib


def lively_case(shape="ar2", Re=1.0, nx=96, ny=40, k_r0=0.03, seed=5):
    """A particle released 0.3 lu above the bottom wall of a shear channel
    with soft bonds and fast kinetics: about 270 formations and ruptures per
    2000 steps."""
    cfg = W.shear_channel(nx, ny, Re, tau=0.9, k_f=0.85, k_r0=k_r0, kBT=0.02, seed=seed,
                          sim_id=2, hamaker=1e-6)
    cfg["y_cr"] = 1.0
    p = W.adhesion_particle(cfg, shape, 6.0, x=nx / 3, ligand_density=0.7, sigma=0.02,
                            gap_over_h=0.3 / (ny - 1))
    return cfg, p


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
def test_bond_replay_bit_exact(O, L, storage):
    cfg, p = lively_case()
    o = O.OracleSim(**cfg)
    o.add_particle(**p)
    g = L.Sim(storage=storage, **cfg)
    g.add_particle(**p)
    steps = 2000
    events, prev, bonded = 0, None, 0
    for t in range(steps):
        po = o.particle(0)
        g.set_record(0, xc=po["xc"], yc=po["yc"], theta=po["theta"], u=po["u"], v=po["v"],
                     omega=po["omega"], step=t)
        o.step(1)
        g.step(1)
        bo, ao = o.bonds(0)
        bg, ag = g.bonds(0)
        assert np.array_equal(bo, bg), (
            f"{storage}: bond flags differ at step {t + 1} "
            f"(oracle margins |U-P| {o.particle(0)['margin_p']:.3g}, "
            f"|gap-y_cr| {o.particle(0)['margin_gap']:.3g})")
        np.testing.assert_allclose(ag[bg == 1], ao[bo == 1], rtol=0, atol=1e-12)
        go, gg = o.particle(0), g.particle(0)
        assert gg["n_probing"] == go["n_probing"] and gg["n_bonded"] == go["n_bonded"]
        if prev is not None:
            events += int((bo != prev).sum())
        prev = bo
        bonded += int(bo.sum())
    assert events > 100 and bonded > 0
    g.close()


def free_run_bonds(o, g, steps, label):
    """Steps oracle and GPU side by side and compares the bond flags at every
    step.  Returns (first divergence step or None, final Hamming distance)."""
    first = None
    for t in range(steps):
        o.step(1)
        g.step(1)
        bo, _ = o.bonds(0)
        bg, _ = g.bonds(0)
        if first is None and not np.array_equal(bo, bg):
            first = t + 1
            st = o.particle(0)
            assert min(st["margin_p"], st["margin_gap"]) < NEAR_TIE, (
                f"{label}: bond flags differ at step {first} without a near tie "
                f"(|U-P| {st['margin_p']:.3g}, |gap-y_cr| {st['margin_gap']:.3g})")
    bo, _ = o.bonds(0)
    bg, _ = g.bonds(0)
    ham = int((bo != bg).sum())
    print(f"{label}: first bond divergence {first}, Hamming distance {ham} after {steps} steps")
    return first, ham


@pytest.mark.parametrize("shape", ["circle", "ar3"])
def test_free_run_f32_bonds_every_step(O, L, shape):
    cfg, p = lively_case(shape=shape, Re=0.1, nx=128, ny=48)
    o = O.OracleSim(**cfg)
    o.add_particle(**p)
    g = L.Sim(storage="f32", **cfg)
    g.add_particle(**p)
    first, _ = free_run_bonds(o, g, 1000, f"f32 {shape}")
    if first is None:
        po, pg = o.particle(0), g.particle(0)
        for k in ("xc", "yc", "theta"):
            assert abs(pg[k] - po[k]) < 1e-4, k
    g.close()
