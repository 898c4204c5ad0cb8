"""Serving-loop scheduling on the host (no GPU): admission by memory budget,
quanta that stop at the nearest completion, exact step counts, latency
accounting, and the trace generator's recipe."""
import math

import numpy as np
import pytest

from paper_1808_01448_gb300 import serve, workloads as W


class FakeEngine:
    """Advances a virtual clock by the work of each step call (updates /
    rate) and records what the scheduler asks for."""

    def __init__(self, rate=1e9):
        self.t = 0.0
        self.rate = rate
        self.members = []
        self.steps_done = {}
        self.calls = []
        self.max_active = 0

    def clock(self):
        return self.t

    def create(self, req):
        self.steps_done[req["rid"]] = 0
        self.modes = getattr(self, "modes", {})
        self.modes[req["rid"]] = req.get("stream_mode", "ab")
        return req["rid"]

    def rebuild(self, members):
        self.members = [m[1] for m in members]
        self.max_active = max(self.max_active, len(self.members))

    def step(self, n):
        self.calls.append((n, tuple(self.members)))
        work = 0
        for rid in self.members:
            self.steps_done[rid] += n
            work += self.nodes[rid] * n
        self.t += work / self.rate

    def result(self, h):
        return [{"steps": self.steps_done[h]}]

    def destroy(self, h):
        self.members = [m for m in self.members if m != h]

    def idle(self, s):
        self.t += s


def small_trace(n=12, seed=7, sizes=(64, 128, 256)):
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for rid in range(n):
        t += rng.exponential(0.05)
        nx = int(rng.choice(sizes))
        out.append(dict(rid=rid, arrival_s=t, steps=int(rng.integers(10, 400)),
                        storage="f32" if rid % 2 else "f16",
                        config=dict(nx=nx, ny=nx // 4), particles=[{}]))
    return out


def run(trace, **kw):
    eng = FakeEngine(rate=kw.pop("rate", 2e7))
    eng.nodes = {r["rid"]: r["config"]["nx"] * r["config"]["ny"] for r in trace}
    srv = serve.Server(eng, clock=eng.clock, **kw)
    res = srv.run(trace, t0=0.0)
    return eng, srv, res


def test_every_request_gets_exactly_its_steps():
    trace = small_trace()
    eng, srv, res = run(trace, quantum=64)
    assert sorted(r.rid for r in res) == list(range(len(trace)))
    for r in res:
        assert r.particles[0]["steps"] == r.steps
        assert eng.steps_done[r.rid] == r.steps
    assert all(n <= 64 for n, _ in eng.calls)
    assert srv.updates == sum(r["steps"] * r["config"]["nx"] * r["config"]["ny"] for r in trace)


def test_latency_is_arrival_to_result_and_ordered():
    trace = small_trace()
    eng, srv, res = run(trace, quantum=50)
    done = [r.done_s for r in res]
    assert done == sorted(done)
    for r in res:
        assert r.admitted_s >= r.arrival_s - 1e-12
        assert r.done_s > r.admitted_s
        assert r.latency_s == pytest.approx(r.done_s - r.arrival_s)
    p50, p99 = serve.latency_stats(res)
    lat = sorted(r.latency_s for r in res)
    assert p50 == lat[math.ceil(0.5 * len(lat)) - 1]
    assert p99 == lat[-1]


def test_admission_respects_the_memory_budget():
    trace = small_trace(20)
    sizes = {r["rid"]: serve.request_bytes(r) for r in trace}
    budget = 3 * max(sizes.values())
    eng = FakeEngine(rate=1e6)
    eng.nodes = {r["rid"]: r["config"]["nx"] * r["config"]["ny"] for r in trace}
    srv = serve.Server(eng, budget_bytes=budget, quantum=32, clock=eng.clock, in_place="never")
    res = srv.run(trace, t0=0.0)
    assert len(res) == len(trace)
    assert srv.admitted_in_place == 0
    for n, members in eng.calls:
        assert sum(sizes[m] for m in members) <= budget
    # requests are admitted in arrival order
    adm = sorted(res, key=lambda r: r.rid)
    assert all(a.admitted_s <= b.admitted_s for a, b in zip(adm, adm[1:]))


def test_in_place_admission_when_two_buffers_do_not_fit():
    """With in_place="auto" a request whose two population buffers do not
    fit the budget left is admitted with one (in-place streaming) when that
    fits; the memory in use never exceeds the budget, counted per mode."""
    trace = small_trace(20, sizes=(512, 1024))
    ab = {r["rid"]: serve.request_bytes(r, "ab") for r in trace}
    aa = {r["rid"]: serve.request_bytes(r, "aa") for r in trace}
    assert all(aa[k] < ab[k] for k in ab)
    budget = 2 * max(ab.values())
    eng = FakeEngine(rate=1e6)
    eng.nodes = {r["rid"]: r["config"]["nx"] * r["config"]["ny"] for r in trace}
    srv = serve.Server(eng, budget_bytes=budget, quantum=32, clock=eng.clock, in_place="auto")
    res = srv.run(trace, t0=0.0)
    assert len(res) == len(trace)
    assert 0 < srv.admitted_in_place == sum(m == "aa" for m in eng.modes.values())
    for n, members in eng.calls:
        held = sum((aa if eng.modes[m] == "aa" else ab)[m] for m in members)
        assert held <= budget
    # "never" serves the same trace with two buffers each, later on average
    eng2 = FakeEngine(rate=1e6)
    eng2.nodes = eng.nodes
    srv2 = serve.Server(eng2, budget_bytes=budget, quantum=32, clock=eng2.clock, in_place="never")
    res2 = srv2.run(trace, t0=0.0)
    assert set(eng2.modes.values()) == {"ab"}
    assert sum(r.admitted_s for r in res) <= sum(r.admitted_s for r in res2)
    # "always", and a request that names its own mode keeps it
    trace[3]["stream_mode"] = "ab"
    eng3 = FakeEngine(rate=1e6)
    eng3.nodes = eng.nodes
    serve.Server(eng3, budget_bytes=budget, clock=eng3.clock, in_place="always").run(trace, t0=0.0)
    assert eng3.modes[3] == "ab"
    assert all(m == "aa" for k, m in eng3.modes.items() if k != 3)
    with pytest.raises(ValueError):
        serve.Server(eng3, in_place="sometimes")


class HoldingEngine(FakeEngine):
    """A fake engine whose handles hold a known number of bytes (less than
    the admission bound), as the library reports them."""

    def __init__(self, held, **kw):
        super().__init__(**kw)
        self.held = held

    def device_bytes(self, h):
        return self.held[h]


def test_admission_counts_the_bytes_actually_held():
    """Admission checks a request's upper bound against what is left and
    then counts the bytes its handle holds: with handles holding half their
    bound, more requests run together than the bound alone allows, and the
    held bytes of the resident requests never exceed the budget."""
    trace = small_trace(24)
    bound = {r["rid"]: serve.request_bytes(r) for r in trace}
    held = {rid: b // 2 for rid, b in bound.items()}
    budget = 3 * max(bound.values())
    eng = HoldingEngine(held, rate=1e6)
    eng.nodes = {r["rid"]: r["config"]["nx"] * r["config"]["ny"] for r in trace}
    srv = serve.Server(eng, budget_bytes=budget, quantum=32, clock=eng.clock)
    res = srv.run(trace, t0=0.0)
    assert len(res) == len(trace) and srv.used == 0
    for n, members in eng.calls:
        assert sum(held[m] for m in members) <= budget
    plain = FakeEngine(rate=1e6)
    plain.nodes = eng.nodes
    srv2 = serve.Server(plain, budget_bytes=budget, quantum=32, clock=plain.clock)
    srv2.run(trace, t0=0.0)
    assert eng.max_active > plain.max_active


def test_oversized_request_is_rejected():
    trace = small_trace(2)
    eng = FakeEngine()
    eng.nodes = {r["rid"]: 1 for r in trace}
    srv = serve.Server(eng, budget_bytes=1000, clock=eng.clock)
    with pytest.raises(ValueError):
        srv.run(trace, t0=0.0)


def test_max_active_caps_the_batch():
    trace = small_trace(15)
    eng, srv, res = run(trace, quantum=40, max_active=3, rate=1e6)
    assert eng.max_active <= 3
    assert len(res) == len(trace)


def test_batches_continue_while_requests_arrive():
    # a long request keeps running while short ones arrive, join and leave
    trace = [dict(rid=0, arrival_s=0.0, steps=1000, storage="f32",
                  config=dict(nx=64, ny=16), particles=[{}])]
    for i in range(1, 5):
        trace.append(dict(rid=i, arrival_s=0.01 * i, steps=50, storage="f32",
                          config=dict(nx=64, ny=16), particles=[{}]))
    eng, srv, res = run(trace, quantum=100, rate=1e7)
    assert res[-1].rid == 0
    assert any(len(m) > 1 and 0 in m for _, m in eng.calls)


def test_serving_trace_recipe():
    tr = W.serving_trace(200)
    arr = np.array([r["arrival_s"] for r in tr])
    assert np.all(np.diff(arr) > 0)
    assert 200 / arr[-1] == pytest.approx(20.0, rel=0.2)
    for r in tr:
        c = r["config"]
        assert 256 <= c["nx"] <= 2048 and c["nx"] % 32 == 0 and c["ny"] == c["nx"] // 4
        assert 1 <= len(r["particles"]) <= 4
        assert 5000 <= r["steps"] <= 50000
        assert r["storage"] in ("f32", "f16")
        assert 0.3 <= r["particles"][0]["ligand_density"] <= 0.9
        for p in r["particles"]:
            assert p["yc"] - np.min(p["vy"]) > 0          # above the bottom wall
            assert p["yc"] + np.max(p["vy"]) < c["ny"] - 1
            # within the library's particle size limit (LBIB_MAX_PARTICLE_RADIUS)
            assert np.max(np.hypot(p["vx"], p["vy"])) <= 44.0


def test_time_accounting_covers_the_engine_calls():
    """The loop's per-call wall time (create, rebuild, step, result, idle)
    adds up to at most the run's wall time and the step share is the
    engine's virtual stepping time."""
    trace = small_trace(12)
    eng, srv, res = run(trace, rate=2e7)
    t = srv.time_in
    assert set(t) == {"create", "rebuild", "step", "result", "idle"}
    assert t["step"] > 0 and t["idle"] >= 0
    total_work = sum(r["steps"] * r["config"]["nx"] * r["config"]["ny"] for r in trace)
    assert t["step"] == pytest.approx(total_work / 2e7, rel=1e-9)
    assert sum(t.values()) <= max(r.done_s for r in res) + 1e-9
