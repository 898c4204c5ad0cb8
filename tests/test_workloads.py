"""The synthetic inputs (`workloads.py`) against their stated recipe: marker
counts of one element per lattice spacing of perimeter (Sec. "The combined
LB-IB method"), outlines of equal area on the intended curves, the shear
channel's wall speed for its Reynolds number, the thermal energy that makes
the exponent of Eq. 11 one at the critical length, and the seeded design
sweep and serving trace with the sizes and ranges they state.  Host only."""
import math

import numpy as np
import pytest

from paper_1808_01448_gb300 import workloads as W


def shoelace(x, y):
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def test_ramanujan_perimeter_of_a_circle_is_exact():
    for r in (1.0, 7.5, 20.0):
        assert W.ramanujan_perimeter(r, r) == pytest.approx(2.0 * math.pi * r, rel=1e-15)


def test_ramanujan_perimeter_against_the_elliptic_integral():
    # the arc length by the midpoint rule (exponentially accurate for a
    # periodic integrand); Ramanujan's second approximation is within a
    # relative 3 h^5 / 2^17 or so, h = ((a - b) / (a + b))^2
    for a, b in ((28.28, 14.14), (34.64, 11.55)):
        t = (np.arange(200000) + 0.5) * (2.0 * np.pi / 200000)
        exact = np.sum(np.hypot(a * np.sin(t), b * np.cos(t))) * (2.0 * np.pi / 200000)
        h = ((a - b) / (a + b)) ** 2
        assert W.ramanujan_perimeter(a, b) == pytest.approx(exact, rel=3.0 * h ** 5 / 2 ** 17 * 2)


@pytest.mark.parametrize("shape,r,n", [("circle", 10.0, 63), ("circle", 20.0, 126),
                                       ("ar2", 20.0, 137), ("ar3", 20.0, 154)])
def test_marker_counts_follow_the_perimeter(shape, r, n):
    vx, vy = W.particle_outline(shape, r)
    assert len(vx) == len(vy) == n


@pytest.mark.parametrize("shape", ["circle", "ar2", "ar3"])
def test_outlines_have_equal_area_and_lie_on_their_curve(shape):
    r = 20.0
    vx, vy = W.particle_outline(shape, r)
    n = len(vx)
    if shape == "circle":
        np.testing.assert_allclose(np.hypot(vx, vy), r, rtol=1e-14)
        # inscribed regular n-gon
        assert shoelace(vx, vy) == pytest.approx(0.5 * n * r * r * math.sin(2 * math.pi / n),
                                                 rel=1e-12)
    else:
        k = float(shape[2:])
        a, b = r * math.sqrt(k), r / math.sqrt(k)     # semi-major along y
        np.testing.assert_allclose((vx / b) ** 2 + (vy / a) ** 2, 1.0, atol=1e-12)
        # equal arc length between vertices, to the sampling of the curve
        edges = np.hypot(np.diff(np.append(vx, vx[0])), np.diff(np.append(vy, vy[0])))
        assert edges.max() / edges.min() < 1.01
        # a polygon inscribed in the curve, close to its area pi r^2
        assert shoelace(vx, vy) == pytest.approx(math.pi * r * r, rel=2e-3)
        assert shoelace(vx, vy) < math.pi * r * r
    # the lowest vertex lies at most the sagitta of half an element above the
    # lowest point of the curve (radius of curvature there: r, or b^2 / a)
    rho = r if shape == "circle" else b * b / a
    s = W.ramanujan_perimeter(*((r, r) if shape == "circle" else (a, b))) / n
    drop = W.half_height(shape, r) - (-vy.min())
    assert 0.0 <= drop <= 1.01 * (s / 2) ** 2 / (2 * rho)


def test_shear_channel_wall_speed_gives_the_reynolds_number():
    for tau, Re, ny in ((1.0, 0.1, 129), (0.8, 1.0, 64)):
        cfg = W.shear_channel(256, ny, Re, tau=tau)
        nu = (tau - 0.5) / 3.0
        H = ny - 1
        assert cfg["u_top"] * H / nu == pytest.approx(Re, rel=1e-14)
        assert cfg["u_bottom"] == 0.0
        assert cfg["y_cr"] == pytest.approx(W.YCR_OVER_H * H, rel=1e-14)


@pytest.mark.parametrize("ratio", [0.5, 2.0])
def test_thermal_energy_makes_the_eq11_exponent_one_at_the_critical_length(ratio):
    sigma, y_cr, y_eq_ratio = 0.37, 1.7, 0.5
    kBT = W.thermal_energy(sigma, y_cr, y_eq_ratio, ratio)
    d = y_cr - y_eq_ratio * y_cr
    assert abs(sigma - ratio * sigma) * d * d / (2.0 * kBT) == pytest.approx(1.0, rel=1e-14)


def test_adhesion_particle_starts_its_gap_above_the_wall():
    # the curve's lowest point sits the gap above the wall line; the lowest
    # vertex no lower than that and within the sagitta of half an element
    cfg = W.shear_channel(512, 128, 0.1)
    H = cfg["ny"] - 1
    for shape in ("circle", "ar2", "ar3"):
        p = W.adhesion_particle(cfg, shape, 11.0, x=100.0, ligand_density=0.5, sigma=0.1)
        assert p["yc"] - W.half_height(shape, 11.0) == pytest.approx(W.Y0_OVER_H * H, abs=1e-12)
        extra = p["yc"] + p["vy"].min() - W.Y0_OVER_H * H
        assert 0.0 <= extra < 0.05


def test_design_sweep_sizes_and_reproducibility():
    a = W.design_sweep()
    b = W.design_sweep()
    assert len(a) == 72
    seen = set()
    for (ca, pa), (cb, pb) in zip(a, b):
        assert ca == cb
        assert len(pa) == 1
        np.testing.assert_array_equal(pa[0]["vx"], pb[0]["vx"])
        nx, ny = ca["nx"], ca["ny"]
        assert 256 <= nx <= 1024 and nx % 32 == 0
        assert 64 <= ny <= 256 and ny % 8 == 0
        assert pa[0]["xc"] == nx / 4.0
        seen.add(ca["sim_id"])
        # equal area to a circle of diameter 0.18 ny
        r = 0.09 * ny
        assert shoelace(pa[0]["vx"], pa[0]["vy"]) == pytest.approx(math.pi * r * r, rel=1e-2)
    assert seen == set(range(72))
    total = sum(c["nx"] * c["ny"] for c, _ in a)
    assert total == pytest.approx(7.43e6, rel=5e-3)


def test_serving_trace_ranges_and_reproducibility():
    tr = W.serving_trace(200)
    again = W.serving_trace(200)
    t_prev = 0.0
    stores = []
    for r, q in zip(tr, again):
        assert r["arrival_s"] == q["arrival_s"] and r["steps"] == q["steps"]
        assert r["arrival_s"] > t_prev
        t_prev = r["arrival_s"]
        nx, ny = r["config"]["nx"], r["config"]["ny"]
        assert nx % 32 == 0 and 256 <= nx <= 2048 and ny == nx // 4
        assert 1 <= len(r["particles"]) <= 4
        assert 5000 <= r["steps"] <= 50000
        Re = r["config"]["u_top"] * (ny - 1) / ((r["config"]["tau"] - 0.5) / 3.0)
        assert 0.01 - 1e-12 <= Re <= 1.0 + 1e-12
        stores.append(r["storage"])
    assert set(stores) == {"f32", "f16"}
    # Poisson arrivals at 20 per second: the mean gap within a few sigma
    gaps = np.diff([0.0] + [r["arrival_s"] for r in tr])
    assert gaps.mean() == pytest.approx(1.0 / 20.0, rel=0.25)
