"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only -- particle outlines, parameter sets
and random smooth fields -- and none of the method's arithmetic.  Both the
CUDA path and the CPU oracle take what it returns.

Workloads (Sec. "Modeling the adhesion dynamics", Table 1): a channel of
height H (lattice rows) with a fixed bottom wall and a moving top wall
(linear shear, Re = u_max H / nu), particles of equal area -- circles and
ellipses of aspect ratio 2 and 3 with the major axis normal to the wall --
released at rest a gap y_0 = 3e-3 H above the bottom wall, ligand densities
0.3..0.9 and spring constants 1 and 2 (lattice units).
"""
from __future__ import annotations

import math

import numpy as np

NU_PAPER = 1.0 / 6.0          # Table 1: nu_ref in lattice units (tau = 1)
Y0_OVER_H = 3.0e-3            # initial gap
YCR_OVER_H = 6.8e-3           # critical bond length
KF_OVER_KR0 = 8.5e3           # biochemical affinity k_f / k_r0
# Table 1's dimensionless groups, which agree with its SI column:
SIGMA_HAT = {1: 27.8, 2: 55.5}   # sigma / (rho_ref nu_ref^2 / H) for bond strength 1 and 2
HAMAKER_HAT = 1.74e-8            # H_k / (rho_ref nu_ref^2 H)
K_R0 = 1.0e-4                    # reverse rate per step (absolute value not given)
# Lower clamp of the gap in Eq. 12 (lattice units).  With Table 1's Hamaker
# group the wall force is weak against the bonds; clamped at 0.1 it cannot
# hold a bonded particle off the wall (most particles of these workloads
# crossed the wall line within 20k steps), clamped at 1e-3 its growth as
# gap^-5/2 stops every one of them a few thousandths of a node from the wall.
EPS_MIN = 1.0e-3


def bond_sigma(strength: int, H: float, nu: float) -> float:
    """Spring constant in lattice units for bond strength 1 or 2 (rho = 1)."""
    return SIGMA_HAT[strength] * nu * nu / H


def hamaker_lu(H: float, nu: float) -> float:
    return HAMAKER_HAT * nu * nu * H


def thermal_energy(sigma: float, y_cr: float, y_eq_ratio: float = 0.5,
                   sigma_star_ratio: float = 0.5) -> float:
    """k_B T such that the exponent of Eq. 11 has magnitude 1 at the critical
    length: +1 for slip bonds (sigma* < sigma), -1 for catch bonds
    (sigma* > sigma).  For sigma* = sigma (ideal bonds) the exponent is 0 and
    k_B T is taken as if sigma* were sigma / 2."""
    d = (1.0 - y_eq_ratio) * y_cr
    r = abs(1.0 - sigma_star_ratio) or 0.5
    return r * sigma * d * d / 2.0


def ramanujan_perimeter(a: float, b: float) -> float:
    h = ((a - b) / (a + b)) ** 2
    return math.pi * (a + b) * (1.0 + 3.0 * h / (10.0 + math.sqrt(4.0 - 3.0 * h)))


def n_markers(a: float, b: float) -> int:
    """One element per lattice spacing of perimeter."""
    return max(8, int(round(ramanujan_perimeter(a, b))))


def circle_polygon(r: float, n: int):
    t = 2.0 * np.pi * np.arange(n) / n
    return r * np.cos(t), r * np.sin(t)


def ellipse_polygon(ax: float, by: float, n: int, samples: int = 200_000):
    """Counter-clockwise polygon on the ellipse (x/ax)^2 + (y/by)^2 = 1 with
    vertices at equal arc length, starting at (ax, 0)."""
    t = np.linspace(0.0, 2.0 * np.pi, samples + 1)
    x, y = ax * np.cos(t), by * np.sin(t)
    seg = np.hypot(np.diff(x), np.diff(y))
    s = np.concatenate([[0.0], np.cumsum(seg)])
    targets = s[-1] * np.arange(n) / n
    tv = np.interp(targets, s, t)
    return ax * np.cos(tv), by * np.sin(tv)


def particle_outline(shape: str, radius_eq: float, n: int | None = None):
    """Outline of equal area pi * radius_eq^2.  shape: 'circle', 'ar2', 'ar3'
    (or 'arK' for any aspect ratio K); ellipses have the major axis along the
    body y axis, so theta = 0 puts it normal to the wall."""
    if shape == "circle":
        n = n or n_markers(radius_eq, radius_eq)
        return circle_polygon(radius_eq, n)
    k = float(shape[2:])
    a = radius_eq * math.sqrt(k)          # semi-major (body y)
    b = radius_eq / math.sqrt(k)          # semi-minor (body x)
    n = n or n_markers(a, b)
    return ellipse_polygon(b, a, n)


def half_height(shape: str, radius_eq: float) -> float:
    """Extent of the outline below its centroid at theta = 0."""
    if shape == "circle":
        return radius_eq
    return radius_eq * math.sqrt(float(shape[2:]))


def shear_channel(nx: int, ny: int, Re: float, tau: float = 1.0, **extra) -> dict:
    """Linear-shear channel of the paper: Zou-He walls on rows 0 and ny-1
    (H = ny - 1), bottom fixed, top moving at u_max = Re nu / H."""
    nu = (tau - 0.5) / 3.0
    H = ny - 1
    cfg = dict(nx=nx, ny=ny, wall_bottom="zou_he", wall_top="zou_he", tau=tau,
               u_bottom=0.0, u_top=Re * nu / H, y_cr=YCR_OVER_H * H)
    cfg.update(extra)
    return cfg


def adhesion_particle(cfg: dict, shape: str, radius_eq: float, x: float,
                      ligand_density: float, sigma: float, gap_over_h: float = Y0_OVER_H,
                      n: int | None = None) -> dict:
    """Particle at rest with its lowest point gap_over_h * H above the bottom
    wall line, major axis normal to the wall."""
    vx, vy = particle_outline(shape, radius_eq, n)
    H = cfg["ny"] - 1 if cfg.get("wall_bottom", "zou_he") == "zou_he" else cfg["ny"]
    y_wall = 0.0 if cfg.get("wall_bottom", "zou_he") == "zou_he" else -0.5
    yc = y_wall + half_height(shape, radius_eq) + gap_over_h * H
    return dict(vx=vx, vy=vy, xc=x, yc=yc, theta=0.0, rho_p=1.0,
                ligand_density=ligand_density, sigma=sigma)


def adhesion_params(H: float, nu: float, strength: int, sigma_star_ratio: float = 0.5,
                    ycr_over_h: float = YCR_OVER_H) -> dict:
    """Bond and wall-force constants in lattice units for bond strength 1 or
    2: Table 1's dimensionless groups scaled by rho nu^2 / H (spring) and
    rho nu^2 H (Hamaker), k_f / k_r0 = 8.5e3, k_B T from thermal_energy.
    sigma_star_ratio = sigma* / sigma (Eq. 11): 0.5 slip bonds (the paper's
    choice), above 1 catch bonds."""
    sigma = bond_sigma(strength, H, nu)
    y_cr = ycr_over_h * H
    return dict(sigma=sigma, y_cr=y_cr, k_r0=K_R0, k_f=KF_OVER_KR0 * K_R0,
                sigma_star_ratio=sigma_star_ratio,
                kBT=thermal_energy(sigma, y_cr, sigma_star_ratio=sigma_star_ratio),
                hamaker=hamaker_lu(H, nu), eps_min=EPS_MIN)


def single_ellipse_sweep(nx: int = 1024, ny: int = 256, radius_eq: float = 20.0,
                         shapes=("ar2", "ar3"), reynolds=(0.01, 0.1, 1.0),
                         ligand_density: float = 0.7, strength: int = 2,
                         seed: int = 2):
    """Single elliptical particle, aspect ratio 2 and 3, equal area to a circle
    of radius 20, in a 1024 x 256 channel at Re 0.01, 0.1 and 1, ligand
    density 0.7, bond strength 2: one sim per (shape, Re).  Returns a list of
    (config, [particle]) pairs."""
    out = []
    sim_id = 0
    for shape in shapes:
        for Re in reynolds:
            cfg = shear_channel(nx, ny, Re, seed=seed, sim_id=sim_id)
            ap = adhesion_params(ny - 1, (cfg["tau"] - 0.5) / 3.0, strength)
            sigma = ap.pop("sigma")
            cfg.update(ap)
            p = adhesion_particle(cfg, shape, radius_eq, x=nx / 4.0,
                                  ligand_density=ligand_density, sigma=sigma)
            out.append((cfg, [p]))
            sim_id += 1
    return out


def ycr_sweep(ycr_over_h=(3.4e-3, 6.8e-3, 1.36e-2), nx: int = 1024, ny: int = 256,
              shape: str = "ar2", Re: float = 0.1, ligand_density: float = 0.7,
              strength: int = 2, sigma_star_ratio: float = 0.5, seed: int = 7):
    """Elliptical particle (equal area to a circle of radius 20) in the shear
    channel for several critical bond lengths y_cr / H (the paper's Fig. 7
    study; 6.8e-3 is its default), one simulation each; sigma_star_ratio
    above 1 gives catch bonds.  Returns (config, [particle]) pairs."""
    out = []
    for sim_id, ycr in enumerate(ycr_over_h):
        cfg = shear_channel(nx, ny, Re, seed=seed, sim_id=sim_id)
        ap = adhesion_params(ny - 1, (cfg["tau"] - 0.5) / 3.0, strength, sigma_star_ratio, ycr)
        sigma = ap.pop("sigma")
        cfg.update(ap)
        p = adhesion_particle(cfg, shape, 20.0, x=nx / 4.0, ligand_density=ligand_density,
                              sigma=sigma)
        out.append((cfg, [p]))
    return out


def design_sweep(seed: int = 3, shapes=("circle", "ar2", "ar3"),
                 ligand_densities=(0.3, 0.5, 0.7, 0.9), strengths=(1, 2),
                 reynolds=(0.01, 0.1, 1.0)):
    """Batched design sweep: one simulation per (shape, ligand density, bond
    strength, Re), sim_id in that order (72 by default).  Lattice sizes drawn
    with PCG64(seed): nx uniform in {256, 288, ..., 1024}, ny uniform in
    {64, 72, ..., 256}.  Shear channel as in the paper; a circle of diameter
    0.18 ny or an ellipse of equal area, major axis normal to the wall, at
    rest a gap 3e-3 H above the bottom wall, x = nx / 4.  Returns a list of
    (config, [particle]) pairs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    combos = [(sh, rl, st, Re) for sh in shapes for rl in ligand_densities
              for st in strengths for Re in reynolds]
    nxs = rng.integers(0, (1024 - 256) // 32 + 1, size=len(combos)) * 32 + 256
    nys = rng.integers(0, (256 - 64) // 8 + 1, size=len(combos)) * 8 + 64
    out = []
    for sim_id, ((shape, rl, strength, Re), nx, ny) in enumerate(zip(combos, nxs, nys)):
        nx, ny = int(nx), int(ny)
        cfg = shear_channel(nx, ny, Re, seed=seed, sim_id=sim_id)
        ap = adhesion_params(ny - 1, (cfg["tau"] - 0.5) / 3.0, strength)
        sigma = ap.pop("sigma")
        cfg.update(ap)
        p = adhesion_particle(cfg, shape, 0.09 * ny, x=nx / 4.0, ligand_density=rl,
                              sigma=sigma)
        out.append((cfg, [p]))
    return out


def particle_cluster(nx: int = 4096, ny: int = 1024, n_particles: int = 8, Re: float = 1.0,
                     ligand_density: float = 0.5, strength: int = 2, seed: int = 4,
                     r_range=(12.0, 24.0)):
    """Precision-study channel: a shear channel at Re with n_particles
    circles or equal-area ellipses (AR 2 or 3) near the bottom wall.  Drawn
    with PCG64(seed): equal-area radius uniform in r_range, shape uniform over
    {circle, ar2, ar3}, gap between the lowest point and the wall uniform in
    [3e-3 H, 3 r] (and the top of the particle below 3/4 H); x positions rejection-sampled so that neighbouring
    centroids are at least 2.5 (r_i + r_j) / 2 apart and clear of each other's
    extent.  One simulation with several particles: (config, [particles])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cfg = shear_channel(nx, ny, Re, seed=seed, sim_id=0)
    H = ny - 1
    ap = adhesion_params(H, (cfg["tau"] - 0.5) / 3.0, strength)
    sigma = ap.pop("sigma")
    cfg.update(ap)
    shapes = ("circle", "ar2", "ar3")
    placed = []
    parts = []
    tries = 0
    while len(parts) < n_particles:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place the particles")
        r = float(rng.uniform(*r_range))
        shape = shapes[int(rng.integers(0, 3))]
        half_w = r if shape == "circle" else r / math.sqrt(float(shape[2:]))
        # the particle stays at least a quarter of the channel below the top
        room = 0.75 * H - 2.0 * half_height(shape, r)
        if room <= Y0_OVER_H * H:
            continue
        gap = float(rng.uniform(Y0_OVER_H * H, min(3.0 * r, room)))
        x = float(rng.uniform(2.0 * r, nx - 2.0 * r))
        if any(abs(x - px) < max(2.5 * (r + pr) / 2.0, half_w + pw + 2.0)
               for px, pr, pw in placed):
            continue
        p = adhesion_particle(cfg, shape, r, x=x, ligand_density=ligand_density,
                              sigma=sigma, gap_over_h=gap / H)
        placed.append((x, r, half_w))
        parts.append(p)
    return cfg, parts


def serving_trace(n_requests: int = 600, rate: float = 20.0, seed: int = 5,
                  steps_range=(5000, 50000)):
    """Simulation requests for the serving loop, drawn with PCG64(seed):
    Poisson arrivals at `rate` per second; nx = 2^U[8, 11] rounded to a
    multiple of 32, ny = nx / 4; 1-4 particles of aspect ratio U[1, 3]
    (equal-area radius 0.09 ny, at most 20, major axis normal to the wall,
    spread evenly along x near the bottom wall); ligand density U[0.3, 0.9]; bond strength
    1 or 2; Re log-uniform in [0.01, 1]; steps log-uniform in steps_range;
    FP32 or FP16 storage with equal probability.  Returns a list of dicts
    with 'arrival_s', 'steps', 'storage', 'config' and 'particles'."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        nx = int(round(2.0 ** rng.uniform(8.0, 11.0) / 32.0)) * 32
        ny = nx // 4
        k = int(rng.integers(1, 5))
        rl = float(rng.uniform(0.3, 0.9))
        strength = int(rng.integers(1, 3))
        Re = float(10.0 ** rng.uniform(-2.0, 0.0))
        steps = int(round(math.exp(rng.uniform(math.log(steps_range[0]),
                                               math.log(steps_range[1])))))
        storage = "f32" if rng.uniform() < 0.5 else "f16"
        ars = [float(rng.uniform(1.0, 3.0)) for _ in range(k)]
        cfg = shear_channel(nx, ny, Re, seed=seed, sim_id=rid)
        ap = adhesion_params(ny - 1, (cfg["tau"] - 0.5) / 3.0, strength)
        sigma = ap.pop("sigma")
        cfg.update(ap)
        parts = []
        for i, ar in enumerate(ars):
            shape = f"ar{ar:.6f}"
            parts.append(adhesion_particle(cfg, shape, min(0.09 * ny, 20.0),
                                           x=nx * (i + 1) / (k + 1),
                                           ligand_density=rl, sigma=sigma))
        out.append(dict(rid=rid, arrival_s=t, steps=steps, storage=storage, config=cfg,
                        particles=parts))
    return out


def poiseuille_circle(nx: int = 200, ny: int = 50, radius: float = 10.0, tau: float = 0.8,
                      Re: float = 0.1, n: int = 63, ligand_density: float = 0.5,
                      strength: int = 1, seed: int = 1):
    """Single circle of radius 10 in a 200 x 50 body-force Poiseuille channel
    with half-way bounce-back walls (H = ny), centre 1.5 radii above the
    wall, 63 markers.  Re = u_c H / nu with the centre-line speed u_c."""
    nu = (tau - 0.5) / 3.0
    H = ny
    u_c = Re * nu / H
    g = 8.0 * nu * u_c / (H * H)
    cfg = dict(nx=nx, ny=ny, wall_bottom="bounce_back", wall_top="bounce_back", tau=tau,
               gx=g, seed=seed, sim_id=0)
    ap = adhesion_params(H, nu, strength)
    sigma = ap.pop("sigma")
    cfg.update(ap)
    vx, vy = circle_polygon(radius, n)
    p = dict(vx=vx, vy=vy, xc=nx / 4.0, yc=-0.5 + 1.5 * radius, theta=0.0, rho_p=1.0,
             ligand_density=ligand_density, sigma=sigma)
    return cfg, [p]


def smooth_field(rng: np.random.Generator, nx: int, ny: int, amplitude: float,
                 modes: int = 3) -> np.ndarray:
    """Random smooth periodic-in-x field: a few low Fourier modes."""
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    out = np.zeros((ny, nx))
    for _ in range(modes):
        kx = rng.integers(1, 4)
        ky = rng.uniform(0.5, 3.0)
        ph = rng.uniform(0, 2 * np.pi, size=2)
        out += rng.uniform(-1, 1) * np.cos(2 * np.pi * kx * x / nx + ph[0]) * \
            np.cos(np.pi * ky * y / ny + ph[1])
    return amplitude * out / modes


def random_noise(rng: np.random.Generator, shape, amplitude: float) -> np.ndarray:
    return amplitude * rng.uniform(-1.0, 1.0, size=shape)
