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
