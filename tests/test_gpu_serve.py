"""Serving loop on the GPU: requests of different lattices, particle counts
and storage formats join and leave the running batches; each result is bit
for bit the one the request gives when stepped alone."""
import numpy as np
import pytest

from paper_1808_01448_gb300 import serve, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1808_01448_gb300 import build, lbib
    build.build()
    return lbib


def small_requests():
    rng = np.random.Generator(np.random.PCG64(11))
    reqs = []
    t = 0.0
    for rid in range(7):
        nx = int(rng.choice([96, 128, 160]))
        ny = nx // 4 + 8
        k = 1 + rid % 2
        cfg = W.shear_channel(nx, ny, 1.0, tau=0.9, k_f=0.85, k_r0=1e-3, kBT=0.02,
                              seed=11, sim_id=rid, hamaker=1e-6)
        cfg["y_cr"] = 1.0
        parts = []
        for i in range(k):
            p = W.adhesion_particle(cfg, ("circle", "ar2")[(rid + i) % 2], 5.0,
                                    x=nx * (i + 1) / (k + 1), ligand_density=0.7, sigma=0.02,
                                    gap_over_h=0.3 / (ny - 1))
            parts.append(p)
        t += float(rng.exponential(1.0))
        reqs.append(dict(rid=rid, arrival_s=t, steps=int(rng.integers(20, 140)),
                         storage=("f32", "f16")[rid % 2 if rid != 4 else 0], config=cfg,
                         particles=parts))
    return reqs


class RecordingEngine(serve.LbibEngine):
    """Real engine on a virtual clock (one unit per step call) that also keeps
    each finished simulation's populations and bond states."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.t = 0.0
        self.final = {}

    def clock(self):
        return self.t

    def step(self, n):
        super().step(n)
        self.t += 0.37

    def idle(self, s):
        self.t += s

    def create(self, req):
        s = super().create(req)
        s.rid = req["rid"]          # object ids are reused once a simulation is freed
        return s

    def result(self, s):
        parts = super().result(s)
        self.final[s.rid] = (s.populations(), [s.bonds(i)[0] for i in range(len(parts))], parts)
        return parts


def test_served_results_equal_solo_runs(L):
    import torch
    reqs = small_requests()
    streams = {"f32": torch.cuda.Stream(), "f16": torch.cuda.Stream()}
    alloc = L.torch_allocator()
    eng = RecordingEngine(L, {k: v.cuda_stream for k, v in streams.items()}, alloc)
    srv = serve.Server(eng, quantum=16, clock=eng.clock)
    res = srv.run(reqs, t0=0.0)
    assert sorted(r.rid for r in res) == list(range(len(reqs)))
    assert srv.rebuilds > 2           # membership changed while others ran
    by_rid = {r["rid"]: r for r in reqs}
    for r in res:
        req = by_rid[r.rid]
        solo = L.Sim(storage=req["storage"], **req["config"])
        for p in req["particles"]:
            solo.add_particle(**p)
        solo.step(req["steps"])
        f_mix, bonds_mix, parts_mix = eng.final[r.rid]
        np.testing.assert_array_equal(solo.populations(), f_mix)
        assert solo.particles() == parts_mix
        for i in range(len(req["particles"])):
            np.testing.assert_array_equal(solo.bonds(i)[0], bonds_mix[i])
        solo.close()
    eng.close()


def test_in_place_admission_results_equal_solo_runs(L):
    """With a budget that fits the requests' two population buffers for only
    part of the trace, the loop admits some of them with in-place streaming
    (one buffer); their results are still bit for bit the A/B solo runs, and
    the memory the library holds never exceeds the budget."""
    import torch
    reqs = small_requests()
    ab = [serve.request_bytes(r, "ab") for r in reqs]
    aa = [serve.request_bytes(r, "aa") for r in reqs]
    # every request fits alone in place; those whose two buffers do not fit
    # can only be admitted in place
    budget = max(aa)
    must = sum(x > budget for x in ab)
    assert must > 0
    streams = {"f32": torch.cuda.Stream(), "f16": torch.cuda.Stream()}
    eng = RecordingEngine(L, {k: v.cuda_stream for k, v in streams.items()}, L.torch_allocator())
    srv = serve.Server(eng, budget_bytes=budget, quantum=16, clock=eng.clock, in_place="auto")
    peak = 0
    orig_step = eng.step

    def step(n):
        nonlocal peak
        peak = max(peak, srv.used)
        orig_step(n)

    eng.step = step
    res = srv.run(reqs, t0=0.0)
    assert sorted(r.rid for r in res) == list(range(len(reqs)))
    assert srv.admitted_in_place >= must
    assert peak <= budget
    by_rid = {r["rid"]: r for r in reqs}
    for r in res:
        req = by_rid[r.rid]
        solo = L.Sim(storage=req["storage"], **req["config"])
        for p in req["particles"]:
            solo.add_particle(**p)
        solo.step(req["steps"])
        f_mix, bonds_mix, parts_mix = eng.final[r.rid]
        np.testing.assert_array_equal(solo.populations(), f_mix)
        assert solo.particles() == parts_mix
        solo.close()
    eng.close()
