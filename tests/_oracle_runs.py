"""Oracle runs for the long-horizon parity tests, in worker processes
(started with spawn): each returns the per-step bond flags and near-tie
margins of particle 0, and the final fields and particle state."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_case(cfg, parts, steps):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import oracle as O
    o = O.OracleSim(**cfg)
    for p in parts:
        o.add_particle(**p)
    nl = o.particle(0)["nl"]
    bonds = np.zeros((steps, nl), dtype=np.uint8)
    margins = np.zeros((steps, 2))
    for t in range(steps):
        o.step(1)
        bonds[t] = o.bonds(0)[0]
        st = o.particle(0)
        margins[t] = (st["margin_p"], st["margin_gap"])
    r, u, v = o.fields()
    return {"bonds": bonds, "margins": margins, "fields": (r, u, v),
            "particle": o.particle(0)}


def shear_populations(O, cfg):
    """Populations of the developed shear flow between the walls: at each
    row the equilibrium (the oracle's Eq. 2) at rho = 1 and the linear
    profile u = u_top y / (ny - 1) of Zou-He walls, [9][ny][nx]."""
    ny, nx = cfg["ny"], cfg["nx"]
    rows = np.stack([O.equilibrium(1.0, cfg["u_top"] * y / (ny - 1), 0.0) for y in range(ny)])
    return np.ascontiguousarray(np.broadcast_to(rows.T[:, :, None], (9, ny, nx)))


def run_crop(cfg, parts, steps, crop):
    """The oracle for `steps` steps from the developed shear flow; returns
    the fields on the crop window (x0, y0, width, height; x periodic) and
    every particle's state."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import oracle as O
    o = O.OracleSim(**cfg)
    for p in parts:
        o.add_particle(**p)
    o.set_populations(shear_populations(O, cfg))
    o.step(steps)
    x0, y0, w, h = crop
    xs = (np.arange(x0, x0 + w)) % cfg["nx"]
    r, u, v = o.fields()
    cut = tuple(f[y0:y0 + h][:, xs] for f in (r, u, v))
    return {"fields": cut, "particles": [o.particle(k) for k in range(len(parts))],
            "bonds": [o.bonds(k)[0] for k in range(len(parts))]}
