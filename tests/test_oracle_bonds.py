"""Pins of the oracle's stochastic bond kinetics (Eq. 9-11) and of its
counter-based generator."""
import math

import numpy as np
import pytest

from paper_1808_01448_gb300 import workloads as W


def numpy_philox(ctr, key):
    """numpy's Philox4x64-10 bit generator: it increments the 256-bit
    counter before each block, so start one below."""
    c = sum(int(v) << (64 * i) for i, v in enumerate(ctr))
    k = sum(int(v) << (64 * i) for i, v in enumerate(key))
    bg = np.random.Philox(key=k, counter=(c - 1) % (1 << 256))
    return [int(v) for v in bg.random_raw(4)]


def test_philox_matches_numpy_bit_generator(O):
    rng = np.random.default_rng(9)
    cases = [([1, 0, 0, 0], [0, 0]), ([5, 7, 0, 0], [1, 0]),
             ([2 ** 64 - 1, 3, 9, 2 ** 63], [2 ** 64 - 1, 12345])]
    for _ in range(300):
        cases.append(([int(v) for v in rng.integers(0, 2 ** 63, 4, dtype=np.uint64)],
                      [int(v) for v in rng.integers(0, 2 ** 63, 2, dtype=np.uint64)]))
    for ctr, key in cases:
        if sum(ctr) == 0:
            continue
        assert O.philox4x64(ctr, key) == numpy_philox(ctr, key), (ctr, key)


def test_uniforms_are_uniform_and_distinct_per_counter(O):
    us = np.array([O.uniform(1, 0, s, 0, l) for s in range(200) for l in range(100)])
    assert us.min() >= 0.0 and us.max() < 1.0
    assert len(np.unique(us)) == len(us)
    assert us.mean() == pytest.approx(0.5, abs=5 * math.sqrt(1 / 12 / len(us)))
    assert us.var() == pytest.approx(1 / 12, abs=0.01)
    counts, _ = np.histogram(us, bins=20, range=(0, 1))
    e = len(us) / 20
    chi2 = ((counts - e) ** 2 / e).sum()
    assert chi2 < 50.0       # 19 dof: p ~ 1e-4
    # seed, sim id, particle id all change the stream
    a = O.uniform(1, 0, 3, 0, 4)
    assert a != O.uniform(2, 0, 3, 0, 4) and a != O.uniform(1, 1, 3, 0, 4)
    assert a != O.uniform(1, 0, 3, 1, 4)


def test_forward_probability_properties(O):
    """Eq. 10: no probing ligands -> no binding; survival composes
    multiplicatively (a Poisson process); saturates at one."""
    assert O.prob_forward(0.85, 0.0) == 0.0
    for k, N in [(0.85, 0.1), (0.3, 0.5), (2.0, 0.02)]:
        p1 = O.prob_forward(k, N)
        p2 = O.prob_forward(k, 2 * N)
        assert (1 - p2) == pytest.approx((1 - p1) ** 2, rel=1e-13)
        assert 0 < p1 < p2 < 1
    assert O.prob_forward(1e3, 1.0) == 1.0


def test_reverse_probability_properties(O):
    """Eq. 11: at the equilibrium length the rate is k_r0; slip bonds
    (sigma > sigma*) break faster when stretched or compressed, catch bonds
    (sigma < sigma*) slower, and sigma = sigma* removes the load dependence."""
    k0, y_eq, kT = 1e-3, 0.65, 0.1
    base = O.prob_reverse(k0, 2.0, 1.0, y_eq, y_eq, kT)
    assert (1 - base) == pytest.approx(math.exp(-k0), rel=1e-15)
    slip = [O.prob_reverse(k0, 2.0, 1.0, y_eq + d, y_eq, kT) for d in (0.1, 0.3, 0.6)]
    assert base < slip[0] < slip[1] < slip[2]
    assert O.prob_reverse(k0, 2.0, 1.0, y_eq - 0.3, y_eq, kT) == slip[1]
    catch = [O.prob_reverse(k0, 1.0, 2.0, y_eq + d, y_eq, kT) for d in (0.1, 0.3)]
    assert catch[1] < catch[0] < base
    flat = {O.prob_reverse(k0, 1.5, 1.5, y, y_eq, kT) for y in (0.1, 0.65, 1.3)}
    assert flat == {base}
    # the exponent scales with 1 / k_B T
    a = -math.log(1 - O.prob_reverse(k0, 2.0, 1.0, y_eq + 0.3, y_eq, kT)) / k0
    b = -math.log(1 - O.prob_reverse(k0, 2.0, 1.0, y_eq + 0.3, y_eq, 2 * kT)) / k0
    assert math.log(a) == pytest.approx(2 * math.log(b), rel=1e-9)


def frozen_particle_sim(O, steps, **kw):
    cfg = dict(nx=24, ny=14, wall_bottom="bounce_back", wall_top="bounce_back", tau=1.0,
               k_f=0.6, k_r0=0.05, kBT=0.5, y_cr=1.6, y_eq_ratio=0.5, seed=11)
    cfg.update(kw)
    s = O.OracleSim(**cfg)
    vx, vy = W.circle_polygon(4.0, 25)
    s.add_particle(vx, vy, 12.0, -0.5 + 4.0 + 0.25, ligand_density=1.0, sigma=1.0, fixed=True)
    return s, cfg


def test_frozen_particle_bonds_follow_two_state_markov_chains(O):
    """With the particle held fixed, every ligand's bond is a two-state Markov
    chain with constant P_f and P_r: the time-averaged bonded fraction is
    P_f / (P_f + P_r) within the chain's sampling error."""
    T = 6000
    s, cfg = frozen_particle_sim(O, T)
    s.step(1)
    p = s.particle(0)
    n_probe, nl = p["n_probing"], p["nl"]
    assert 2 <= n_probe < nl
    bonded = []
    for _ in range(T):
        s.step(1)
        b, _ = s.bonds(0)
        bonded.append(b.copy())
    bonded = np.array(bonded, dtype=float)
    ex, ey, w, _ = O.lattice()
    vx, vy = W.circle_polygon(4.0, 25)
    mx, my, *_ = O.elements(vx, vy, 12.0, -0.5 + 4.25, 0.0)
    gap = my + 0.5
    probing = gap < cfg["y_cr"]
    assert probing.sum() == n_probe
    Pf = O.prob_forward(cfg["k_f"], n_probe / nl)
    y_eq = cfg["y_eq_ratio"] * cfg["y_cr"]
    tot_mean, tot_var = 0.0, 0.0
    for l in np.nonzero(probing)[0]:
        Pr = O.prob_reverse(cfg["k_r0"], 1.0, 0.5, gap[l], y_eq, cfg["kBT"])
        pi = Pf / (Pf + Pr)
        lam = 1 - Pf - Pr
        tot_mean += pi
        tot_var += pi * (1 - pi) * (1 + lam) / (1 - lam) / T
    observed = bonded[:, probing].mean(axis=0).sum()
    assert abs(observed - tot_mean) < 5 * math.sqrt(tot_var)
    assert np.all(bonded[:, ~probing] == 0)


def test_no_bonds_without_receptors_or_ligands(O):
    s, _ = frozen_particle_sim(O, 0, receptor_bottom=0.0)
    s.step(300)
    assert s.bonds(0)[0].sum() == 0 and s.particle(0)["n_probing"] == 0
    cfg = dict(nx=24, ny=14, tau=1.0, k_f=0.6, y_cr=1.6)
    s = O.OracleSim(**cfg)
    vx, vy = W.circle_polygon(4.0, 25)
    s.add_particle(vx, vy, 12.0, 3.75, ligand_density=0.0, fixed=True)
    s.step(300)
    assert s.bonds(0)[0].sum() == 0 and s.particle(0)["n_ligands"] == 0


def test_ligands_are_evenly_spread(O):
    s = O.OracleSim(nx=40, ny=30)
    vx, vy = W.circle_polygon(8.0, 50)
    for rho_l in (0.3, 0.5, 0.7, 0.9, 1.0):
        pid = s.add_particle(vx, vy, 20.0, 15.0, ligand_density=rho_l)
        n = s.particle(pid)["n_ligands"]
        assert n == math.floor(50 * rho_l + 1e-9)
