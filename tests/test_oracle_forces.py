"""Pins of the oracle's wall force (Eq. 12), bond spring force and moment
(Eq. 9 with the anchor reading: the bond runs from the ligand's element
centroid to an anchor fixed on the wall line at formation) and of the
direct-forcing factor of the IB step (Sec. "The combined LB-IB method",
Favier et al.: F_l = 2 rho_l (U^d_l - u*_l), spread with eps_l = S_l).

Each expected value is computed here from the polygon's vertices, not from
the oracle's own element routine, so that a wrong exponent, sign, wall or
factor in the oracle fails."""
import math

import numpy as np
import pytest

from paper_1808_01448_gb300 import workloads as W


def element_centroids(vx, vy, xc, yc, theta):
    """Midpoints and lengths of the polygon's edges at a pose, from the
    rotated vertices."""
    c, s = math.cos(theta), math.sin(theta)
    ax = xc + c * vx - s * vy
    ay = yc + s * vx + c * vy
    bx, by = np.roll(ax, -1), np.roll(ay, -1)
    return 0.5 * (ax + bx), 0.5 * (ay + by), np.hypot(bx - ax, by - ay)


def shoelace(vx, vy):
    return 0.5 * float(np.sum(vx * np.roll(vy, -1) - np.roll(vx, -1) * vy))


def eq12(H, r, gap):
    return H / (8.0 * math.sqrt(2.0)) * math.sqrt(r / gap ** 5)


# wall lines: (bottom y, top y minus (ny - 1)); Zou-He walls on the node rows, half-way
# bounce-back half a node beyond them
WALL_LINES = {"zou_he": (0.0, 0.0), "bounce_back": (-0.5, 0.5)}


@pytest.mark.parametrize("walls", ["zou_he", "bounce_back"])
@pytest.mark.parametrize("where", ["bottom", "top", "both", "clamped"])
def test_wall_force_closed_form(O, walls, where):
    """Eq. 12 on a fixed polygon at a known smallest element gap:
    F_w = H_k / (8 sqrt 2) sqrt(r / eps^5) along the wall normal into the
    fluid (+y off the bottom wall, -y off the top), r = sqrt(A / pi), eps the
    smallest element-centroid gap clamped below by eps_min."""
    ny = 24 if where == "both" else 40
    H, eps_min = 3e-3, 0.1
    cfg = dict(nx=48, ny=ny, wall_bottom=walls, wall_top=walls, tau=0.8, hamaker=H,
               eps_min=eps_min, k_f=0.0, k_r0=0.0)
    vx, vy = W.particle_outline("ar2", 5.0)
    theta = 0.35
    yb = WALL_LINES[walls][0]
    yt = ny - 1 + WALL_LINES[walls][1]
    mx, my, _ = element_centroids(vx, vy, 0.0, 0.0, theta)
    lo, hi = my.min(), my.max()
    if where == "bottom":
        yc = yb + 0.73 - lo
    elif where == "top":
        yc = yt - 0.41 - hi
    elif where == "clamped":
        yc = yb + 0.02 - lo          # below eps_min: the clamp applies
    else:
        # a channel narrow enough that both gaps matter
        yc = 0.5 * (yb + yt) - 0.5 * (lo + hi) + 0.3
    s = O.OracleSim(**cfg)
    s.add_particle(vx, vy, 23.6, yc, theta=theta, ligand_density=0.0, sigma=0.0, fixed=True)
    s.step(1)
    p = s.particle(0)
    _, my, _ = element_centroids(vx, vy, 23.6, yc, theta)
    eb = max(float((my - yb).min()), eps_min)
    et = max(float((yt - my).min()), eps_min)
    r = math.sqrt(shoelace(vx, vy) / math.pi)
    expect = eq12(H, r, eb) - eq12(H, r, et)
    assert p["Fw"][0] == 0.0
    assert p["Fw"][1] == pytest.approx(expect, rel=1e-12)
    if where == "bottom":
        assert expect > 0 and eb == pytest.approx(0.73, abs=1e-12)
    if where == "top":
        assert expect < 0
    if where == "clamped":
        assert eb == eps_min


@pytest.mark.parametrize("walls", ["zou_he", "bounce_back"])
def test_bond_spring_force_and_moment(O, walls):
    """Eq. 9 on a fixed particle with two bonds placed by hand (one to each
    wall), no formation (k_f = 0) and no rupture (k_r0 = 0): each bond pulls
    its ligand's element centroid X_l toward its anchor with magnitude
    sigma (y_l - y_eq), y_l = |anchor - X_l|, and adds the moment
    (X_l - X_c) x f about the centroid."""
    ny = 30
    sigma, y_cr, y_eq_ratio = 0.37, 2.0, 0.5
    cfg = dict(nx=48, ny=ny, wall_bottom=walls, wall_top=walls, tau=0.8, k_f=0.0, k_r0=0.0,
               kBT=0.1, y_cr=y_cr, y_eq_ratio=y_eq_ratio, receptor_bottom=1.0, receptor_top=1.0)
    vx, vy = W.particle_outline("ar3", 4.0)
    xc, yc, theta = 21.3, 13.7, 0.6
    s = O.OracleSim(**cfg)
    s.add_particle(vx, vy, xc, yc, theta=theta, ligand_density=1.0, sigma=sigma, fixed=True)
    n = len(vx)
    mx, my, _ = element_centroids(vx, vy, xc, yc, theta)
    lb, lt = int(np.argmin(my)), int(np.argmax(my))
    bond = np.zeros(n, np.uint8)
    ax = np.zeros(n)
    aw = np.zeros(n, np.int8)
    bond[[lb, lt]] = 1
    ax[lb] = mx[lb] + 0.83         # anchors off to the side: both components non-zero
    ax[lt] = mx[lt] - 1.21
    aw[lt] = 1
    s.set_bonds(0, bond, ax, aw)
    s.step(1)
    p = s.particle(0)
    yb = WALL_LINES[walls][0]
    yt = ny - 1 + WALL_LINES[walls][1]
    F = np.zeros(2)
    M = 0.0
    for l, wy in ((lb, yb), (lt, yt)):
        d = np.array([ax[l] - mx[l], wy - my[l]])
        y = float(np.linalg.norm(d))
        f = sigma * (y - y_eq_ratio * y_cr) * d / y
        F += f
        M += (mx[l] - xc) * f[1] - (my[l] - yc) * f[0]
    assert p["n_bonded"] == 2
    np.testing.assert_allclose(p["Fb"], F, rtol=1e-12, atol=1e-15)
    assert p["Mb"] == pytest.approx(M, rel=1e-12)
    b, a, w = s.bonds(0, walls=True)
    assert np.array_equal(b, bond) and np.array_equal(w, aw) and np.array_equal(a, ax)


def test_direct_forcing_factor(O):
    """The direct-forcing amplitude: with markers whose 4 x 4 supports do
    not overlap (midpoints of a square of side 8) in a uniform flow u0 at
    rho = 1, one spread of F_l = 2 rho (U^d_l - u*_l) with eps_l = S_l
    changes the Guo half-step velocity interpolated at each marker by exactly
    (U^d_l - u0) S_l sum_k phi_k(X_l)^2 (the interpolation of the field
    spread from the marker alone).  A factor 1 instead of 2, or a missing
    eps_l, fails."""
    nx = ny = 48
    u0 = np.array([3e-3, -1.2e-3])
    cfg = dict(nx=nx, ny=ny, wall_bottom="periodic", wall_top="periodic", tau=0.9)
    feq = O.equilibrium(1.0, u0[0], u0[1])
    f = np.broadcast_to(feq[:, None, None], (9, ny, nx)).copy()
    side = 8.0
    vx = 0.5 * side * np.array([1.0, -1.0, -1.0, 1.0])     # counter-clockwise square
    vy = 0.5 * side * np.array([-1.0, -1.0, 1.0, 1.0])
    xc, yc = 24.37, 23.61
    s = O.OracleSim(**cfg)
    s.add_particle(vx, vy, xc, yc, theta=0.0, ligand_density=0.0, sigma=0.0, fixed=True)
    s.set_populations(f)
    fx, fy = s.ib_force()
    mx, my, S = element_centroids(vx, vy, xc, yc, 0.0)
    c = O.make_config(**cfg)
    Ix = O.interp(c, fx, mx, my)
    Iy = O.interp(c, fy, mx, my)
    for l in range(4):
        _, _, phi = O.mls_shape(c, mx[l], my[l])
        q = S[l] * float((phi ** 2).sum())
        assert 0.2 < q / S[l] < 1.0
        # Guo half-step velocity change: I_l[f_ib] / (2 rho), rho = 1; U^d = 0
        assert Ix[l] / 2.0 == pytest.approx(-u0[0] * q, rel=1e-12)
        assert Iy[l] / 2.0 == pytest.approx(-u0[1] * q, rel=1e-12)
    # the total spread force: sum_l eps_l F_l (partition of unity)
    assert fx.sum() == pytest.approx(-2.0 * u0[0] * S.sum(), rel=1e-12)


def test_near_tie_margins(O):
    """The oracle's near-tie diagnostics after a bond step: the smallest
    |gap - y_cr| over the ligands' probing tests equals the one computed
    here from the element centroids (a fixed particle, receptors on the
    bottom wall only)."""
    cfg = dict(nx=48, ny=30, wall_bottom="zou_he", wall_top="zou_he", tau=0.8, k_f=0.5,
               k_r0=1e-3, kBT=0.1, y_cr=1.5, receptor_bottom=1.0, receptor_top=0.0)
    vx, vy = W.particle_outline("circle", 5.0)
    s = O.OracleSim(**cfg)
    s.add_particle(vx, vy, 20.2, 6.1, theta=0.0, ligand_density=1.0, sigma=0.01, fixed=True)
    s.step(1)
    p = s.particle(0)
    _, my, _ = element_centroids(vx, vy, 20.2, 6.1, 0.0)
    assert p["margin_gap"] == pytest.approx(float(np.abs(my - 1.5).min()), abs=1e-14)
    assert 0 <= p["margin_p"] < 1
