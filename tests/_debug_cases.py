"""Cases run under both library builds by test_gpu_debug.py: writes the
populations and particle states they end with to an .npz (argv[1])."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1808_01448_gb300 import lbib as L  # noqa: E402
from paper_1808_01448_gb300 import workloads as W  # noqa: E402


def adhesion(nx, ny, shape, sim_id):
    cfg = W.shear_channel(nx, ny, 1.0, tau=0.9, k_f=0.85, k_r0=0.03, kBT=0.02, seed=5,
                          sim_id=sim_id, hamaker=1e-6)
    cfg["y_cr"] = 1.0
    return cfg, W.adhesion_particle(cfg, shape, 6.0, x=nx / 3, ligand_density=0.7, sigma=0.02,
                                    gap_over_h=0.3 / (ny - 1))


def main(out):
    res = {}
    # FP32 and FP16 batches (bulk, near-box and particle passes, vector path)
    for st in ("f32", "f16", "f64"):
        sims = []
        for k, (nx, ny, shape) in enumerate(((96, 40, "ar2"), (128, 48, "circle"))):
            cfg, p = adhesion(nx, ny, shape, k)
            s = L.Sim(storage=st, **cfg)
            s.add_particle(**p)
            sims.append(s)
        b = L.Batch(sims)
        b.step(45)
        b.synchronize()
        for k, s in enumerate(sims):
            res[f"{st}_{k}_pop"] = s.populations()
            res[f"{st}_{k}_x"] = np.array([s.particle(0)[q] for q in ("xc", "yc", "theta")])
        b.close()
    # body-force channel in 16-bit storage (the forced collision of the
    # bulk pass, paired in the release build, node by node in the debug one)
    for st in ("f16", "bf16"):
        cfg, parts = W.poiseuille_circle(Re=5.0)
        s = L.Sim(storage=st, **cfg)
        s.add_particle(**parts[0])
        b = L.Batch([s])
        b.step(30)
        b.synchronize()
        res[f"body_{st}_pop"] = s.populations()
        b.close()
    # a particle carried across work tiles and around the periodic y
    # boundary (the debug build checks the bulk pass's near-box counts)
    for st in ("f32", "f16"):
        cfg = dict(nx=96, ny=64, wall_bottom="periodic", wall_top="periodic", tau=0.8, gy=2e-4,
                   hamaker=0.0, seed=3, sim_id=0)
        vx, vy = W.circle_polygon(6.0, 40)
        s = L.Sim(storage=st, **cfg)
        s.add_particle(vx=vx, vy=vy, xc=40.0, yc=50.0, theta=0.0, rho_p=1.0,
                       ligand_density=0.0, sigma=0.02)
        # a lattice with rows wider than a tile, the box across the x edge
        cfg2 = dict(cfg, nx=2048, ny=48, sim_id=1)
        s2 = L.Sim(storage=st, **cfg2)
        s2.add_particle(vx=vx, vy=vy, xc=2044.0, yc=30.0, theta=0.0, rho_p=1.0,
                        ligand_density=0.0, sigma=0.02)
        b = L.Batch([s, s2])
        b.step(400)
        b.synchronize()
        res[f"rise_{st}_pop"] = s.populations()
        res[f"rise_{st}_y"] = np.array([s.particle(0)["yc"]])
        res[f"rise2_{st}_pop"] = s2.populations()
        res[f"rise2_{st}_y"] = np.array([s2.particle(0)["yc"], s2.particle(0)["xc"]])
        b.close()
    # copy-engine staging variants of the bulk pass (single stage, pipeline)
    for v in (4, 5):
        for st in ("f32", "f16"):
            cfg, p = adhesion(160, 48, "ar3", 7)
            s = L.Sim(storage=st, **cfg)
            s.add_particle(**p)
            b = L.Batch([s])
            b.set_variant(v)
            b.step(20)
            b.synchronize()
            res[f"tma{v}_{st}_pop"] = s.populations()
            b.close()
    print(L.version())
    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1])
