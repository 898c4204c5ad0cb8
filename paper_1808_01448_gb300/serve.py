"""Serving loop: continuous batching of simulation requests on one GPU.

Requests (a channel, its particles, a step count and a storage format)
arrive over time.  The loop admits them while their device memory fits a
budget (a request is admitted when an upper bound of its memory fits what
is left, and then counts with the bytes the library actually allocated for
it, lbib_device_bytes; a request whose two population buffers do not fit is
admitted with in-place streaming, one buffer, when that fits), keeps every
admitted simulation resident, and steps all of them
together: one batch per storage format (members of a batch share one
lattice launch and one particle launch per step, see lbib_batch_*), each on
its own stream so that the two batches overlap on the device.  Batches are
rebuilt only when membership changes.  Each round advances every member by
the same number of steps, at most `quantum` and never past the nearest
completion, so a request finishes exactly at its step count; it is then read
back (particle states and bond counts), freed, and its latency (arrival to
result) recorded.  A simulation's arithmetic does not depend on the batch it
is stepped in, so every result is bit for bit the one it would have alone.

The scheduling logic (admission, quanta, completion, latency accounting) is
independent of the device: `Server` drives an engine object, and
`LbibEngine` is the one that runs the library.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

BYTES_PER_VALUE = {"f32": 4, "f16": 2, "bf16": 2, "f64": 8}


def request_bytes(req, stream_mode: str | None = None) -> int:
    """Device memory of a request: its population buffers (two with A/B
    streaming, one in place) plus a generous allowance for particle
    structs, geometry and force tiles."""
    c = req["config"]
    mode = stream_mode or req.get("stream_mode", "ab")
    buffers = 1 if mode == "aa" else 2
    pops = buffers * 9 * c["nx"] * c["ny"] * BYTES_PER_VALUE[req["storage"]]
    return pops + (1 << 20) * (1 + len(req["particles"]))


@dataclass
class Result:
    rid: int
    arrival_s: float
    admitted_s: float
    done_s: float
    steps: int
    nodes: int
    particles: list = field(default_factory=list)

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


class Server:
    """Continuous-batching scheduler.

    engine: object with create(req) -> handle, step(handles_by_storage,
      nsteps) (enqueue nsteps on every handle, grouped by storage, and wait),
      result(handle) -> list of particle states, destroy(handle), and
      optionally device_bytes(handle) -> the bytes the handle holds.
    budget_bytes: admission limit on the device memory of the active
      requests: a request is admitted when request_bytes (an upper bound)
      fits what is left, and is then counted with device_bytes of its
      handle (request_bytes when the engine has no device_bytes).
    in_place: "auto" admits a request whose A/B form does not fit the budget
      left with in-place streaming (one population buffer: half the memory,
      slower lattice pass) when that fits; "never" waits for A/B room;
      "always" admits every request in place.  A request that names its own
      stream_mode keeps it.
    quantum: largest number of steps between two scheduling decisions.
    max_active: optional cap on the number of resident simulations.
    clock: callable returning seconds (wall clock by default); tests pass a
      virtual clock.
    """

    def __init__(self, engine, budget_bytes: int = 150 << 30, quantum: int = 1000,
                 max_active: int | None = None, clock=None, in_place: str = "auto"):
        if in_place not in ("auto", "never", "always"):
            raise ValueError("in_place must be 'auto', 'never' or 'always'")
        self.engine = engine
        self.budget = int(budget_bytes)
        self.in_place = in_place
        self.admitted_in_place = 0
        self.quantum = int(quantum)
        self.max_active = max_active
        self.clock = clock or time.perf_counter
        self.active = {}          # rid -> [req, handle, remaining, admitted_s]
        self.used = 0
        self.results: list[Result] = []
        self.rounds = 0
        self.rebuilds = 0
        self.updates = 0
        # wall time (clock units) spent in each engine call
        self.time_in = {"create": 0.0, "rebuild": 0.0, "step": 0.0, "result": 0.0, "idle": 0.0}

    def _timed(self, what, fn, *args):
        t = self.clock()
        out = fn(*args)
        self.time_in[what] += self.clock() - t
        return out

    def _admit(self, waiting, now):
        admitted = False
        while waiting and waiting[0][0] <= now:
            _, rid, req = waiting[0]
            modes = [req["stream_mode"]] if "stream_mode" in req else (
                ["aa"] if self.in_place == "always" else
                ["ab", "aa"] if self.in_place == "auto" else ["ab"])
            if request_bytes(req, modes[-1]) > self.budget:
                raise ValueError(f"request {rid} needs {request_bytes(req, modes[-1])} bytes, "
                                 "above the budget")
            fits = [m for m in modes if self.used + request_bytes(req, m) <= self.budget]
            if not fits:
                break
            mode = fits[0]
            need = request_bytes(req, mode)
            if self.max_active is not None and len(self.active) >= self.max_active:
                break
            heapq.heappop(waiting)
            h = self._timed("create", self.engine.create, dict(req, stream_mode=mode))
            self.admitted_in_place += mode == "aa"
            held = need
            if hasattr(self.engine, "device_bytes"):
                held = int(self.engine.device_bytes(h))
                if held > need:
                    raise RuntimeError(f"request {rid} holds {held} bytes, above its bound {need}")
            self.active[rid] = [req, h, int(req["steps"]), now, held]
            self.used += held
            admitted = True
        return admitted

    def run(self, requests, t0: float | None = None):
        """Serve `requests` (each with 'rid', 'arrival_s' relative to t0,
        'steps', 'storage', 'config', 'particles'); returns the results in
        completion order."""
        t0 = self.clock() if t0 is None else t0
        waiting = [(r["arrival_s"], r["rid"], r) for r in requests]
        heapq.heapify(waiting)
        dirty = True
        while waiting or self.active:
            now = self.clock() - t0
            if self._admit(waiting, now):
                dirty = True
            if not self.active:
                # idle until the next arrival
                nxt = waiting[0][0]
                self._timed("idle", self.engine.idle, max(0.0, nxt - now))
                continue
            if dirty:
                self._timed("rebuild", self.engine.rebuild,
                            [(rid, v[1], v[0]["storage"]) for rid, v in self.active.items()])
                self.rebuilds += 1
                dirty = False
            q = min(self.quantum, min(v[2] for v in self.active.values()))
            self._timed("step", self.engine.step, q)
            self.rounds += 1
            now = self.clock() - t0
            finished = [rid for rid, v in self.active.items() if v[2] == q]
            for rid, v in self.active.items():
                v[2] -= q
                c = v[0]["config"]
                self.updates += q * c["nx"] * c["ny"]
            for rid in finished:
                req, h, _, adm, held = self.active.pop(rid)
                parts = self._timed("result", self.engine.result, h)
                self._timed("result", self.engine.destroy, h)
                self.used -= held
                c = req["config"]
                self.results.append(Result(rid, req["arrival_s"], adm, now, int(req["steps"]),
                                           c["nx"] * c["ny"], parts))
            if finished:
                dirty = True
        return self.results


def latency_stats(results):
    """p50 / p99 latency (s) over the results, nearest-rank percentiles."""
    lat = sorted(r.latency_s for r in results)
    if not lat:
        return None, None

    def pct(p):
        k = max(0, min(len(lat) - 1, int(-(-p * len(lat) // 100)) - 1))
        return lat[k]

    return pct(50), pct(99)


class LbibEngine:
    """Engine of the serving loop on the library: one batch per storage
    format, each on its own CUDA stream; device memory from the allocator
    hook (PyTorch's caching allocator when given), so that freeing a
    finished simulation does not synchronise the device."""

    def __init__(self, lbib, streams: dict, allocator=None):
        self.L = lbib
        self.streams = streams          # storage -> cudaStream_t (int)
        self.alloc = allocator
        self.batches = {}               # storage -> Batch
        self.sims = {}                  # handle id -> Sim
        self.variants = {}              # storage -> tuned lattice-pass variant

    def create(self, req):
        st = req["storage"]
        s = self.L.Sim(storage=st, stream=self.streams[st], allocator=self.alloc,
                       stream_mode=req.get("stream_mode", "ab"), **req["config"])
        for p in req["particles"]:
            s.add_particle(**p)
        self.sims[id(s)] = s
        return s

    def rebuild(self, members):
        # only the storage groups whose membership changed get a new batch
        groups = {}
        for _, s, st in members:
            groups.setdefault(st, []).append(s)
        for st in list(self.batches):
            b = self.batches[st]
            if st not in groups or [id(x) for x in b.sims] != [id(x) for x in groups[st]]:
                b.close()
                del self.batches[st]
        for st, ss in groups.items():
            if st not in self.batches:
                b = self.L.Batch(ss)
                # the lattice-pass variant is tuned on the first batch of each
                # storage format and reused for the later ones
                # (a batch with an in-place member has nothing to time)
                if st in self.variants:
                    b.set_variant(self.variants[st])
                else:
                    v, ms = b.autotune(10)
                    if any(ms):
                        self.variants[st] = v
                self.batches[st] = b

    def step(self, n):
        for b in self.batches.values():
            b.step(n)                   # enqueue on every stream first
        for b in self.batches.values():
            b.synchronize()

    def result(self, s):
        return s.particles()

    def device_bytes(self, s):
        return s.device_bytes()

    def destroy(self, s):
        # the batch holding s is rebuilt before the next step
        for st, b in list(self.batches.items()):
            if any(x is s for x in b.sims):
                b.close()
                del self.batches[st]
        self.sims.pop(id(s), None)
        s.close()

    def idle(self, seconds):
        time.sleep(min(seconds, 0.01))

    def close(self):
        for b in self.batches.values():
            b.close()
        self.batches = {}
        for s in self.sims.values():
            s.close()
        self.sims = {}
