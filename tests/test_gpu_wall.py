"""No particle crosses the wall (Eq. 12, Sec. "Wall-particle interaction").

Under the workloads' constants (Table 1's dimensionless groups for the
springs and the Hamaker constant) the bonds dominate the wall force; with
the gap of Eq. 12 clamped at 1e-3 lattice units its gap^-5/2 growth still
keeps every bonded particle on the fluid side of the wall line.  The six
1024 x 256 channels and the 72-channel design sweep are stepped 5000 steps;
every 500 steps each particle's smallest element-centroid gap to the bottom
wall line (the paper's y_min) must be positive, and particles must bond."""
import numpy as np
import pytest

from paper_1808_01448_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1808_01448_gb300 import build, lbib
    build.build()
    return lbib


@pytest.mark.parametrize("name", ["ellipse6", "sweep72"])
def test_bonded_particles_stay_off_the_wall(L, name):
    cases = W.single_ellipse_sweep() if name == "ellipse6" else W.design_sweep()
    sims = []
    for cfg, parts in cases:
        assert cfg["eps_min"] == W.EPS_MIN
        s = L.Sim(storage="f32", **cfg)
        for p in parts:
            s.add_particle(**p)
        sims.append(s)
    b = L.Batch(sims)
    worst, bonded = np.inf, 0
    for _ in range(10):
        b.step(500)
        for row, (cfg, _) in zip(b.particles(), cases):
            gap = row[0]["gap_bottom"]
            assert gap > 0, f"{name}: a particle crossed the bottom wall line (gap {gap:.3g})"
            worst = min(worst, gap / (cfg["ny"] - 1))
            bonded += row[0]["n_bonded"]
    print(f"{name}: smallest y_min / H over 5000 steps {worst:.3e}, "
          f"{bonded / (10 * len(sims)):.2f} bonds per particle on average")
    assert bonded > 0
    b.close()
    for s in sims:
        s.close()
