"""Throughput of the LB-IB-MLS adhesion step on GB300 (one JSON line).

Workload (default): the batched design sweep, 72 independent channels
(shape circle / ellipse AR2 / AR3 x ligand density {0.3, 0.5, 0.7, 0.9} x
bond strength {1, 2} x Re {0.01, 0.1, 1.0}), lattices drawn from 256 x 64 to
1024 x 256 (7.43 M nodes in all), one particle each, FP32 populations with
FP64 MLS solves and rigid-body update, all stepped together (per step one
bulk lattice launch, one near-box launch and one particle launch, replayed
from CUDA graphs).  A "step" is one time step of all 72.  The inputs are
larger than L2: 535 MB of FP32 populations (two buffers) against a 129 MiB
L2, 268 MB in FP16 / BF16, so no flush is needed between steps.

Metric: aggregate MLUPS = sum(nx * ny) * steps / time, with the fraction of
the HBM roofline at 72 B per FP32 lattice update.  Under torchrun every rank
runs the same 72 simulations on its own GPU (independent replicas, no
collective on the data path); value is the total over ranks.

--workload ellipse6 times the six 1024 x 256 channels instead (their 113 MB
of populations fit in L2, which the line's config says).  --impl reference
times the FP64 CPU oracle on a sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_UPDATE = {"f32": 72, "f64": 144, "f16": 36, "bf16": 36}
WORKLOADS = {
    "sweep72": ("batched design sweep: 72 sims (circle/AR2/AR3 x ligand {0.3,0.5,0.7,0.9} x "
                "sigma {1,2} x Re {0.01,0.1,1}), lattices 256x64..1024x256, 7.43 M nodes, "
                "one particle each", "256x64..1024x256"),
    "ellipse6": ("single ellipse AR2/AR3 x Re{0.01,0.1,1}, 1024x256 D2Q9, ligand 0.7, sigma 2, "
                 "6 sims batched", "1024x256"),
}


def workload_cases(name):
    from paper_1808_01448_gb300 import workloads as W
    return W.design_sweep() if name == "sweep72" else W.single_ellipse_sweep()


def wall_report(batch, name, steps):
    """The particles' smallest element-centroid gap to the bottom wall line
    (the paper's y_min, Eq. 12), over the channel height, after the run;
    a particle past the wall line has a negative gap."""
    H = [c["ny"] - 1 if c.get("wall_bottom", "zou_he") == "zou_he" else c["ny"]
         for c, _ in workload_cases(name)]
    gaps, bonded = [], 0
    for h, row in zip(H, batch.particles()):
        for p in row:
            gaps.append(p["gap_bottom"] / h)
            bonded += p["n_bonded"] > 0
    return {"y_min_over_h": min(gaps), "y_min_over_h_median": sorted(gaps)[len(gaps) // 2],
            "crossed": sum(g <= 0 for g in gaps), "bonded_particles": bonded,
            "particles": len(gaps), "after_steps": steps}


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def lattice_kernel_sha():
    h = hashlib.sha256()
    for rel in ("paper_1808_01448_gb300/csrc/lbib_lattice.cu",
                "paper_1808_01448_gb300/csrc/lbib_internal.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(storage):
    """DRAM bytes per lattice-kernel launch from the committed ncu summary,
    if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "lattice_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(storage)
    if not e or e.get("kernel_sha") != lattice_kernel_sha():
        return None
    return e.get("bytes_per_launch_full_workload")


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"lbib_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def build_workload(L, W, storage, stream, allocator, rounding="stochastic", name="sweep72"):
    sims = []
    for cfg, parts in workload_cases(name):
        s = L.Sim(storage=storage, stream=stream, allocator=allocator, rounding=rounding, **cfg)
        for p in parts:
            s.add_particle(**p)
        sims.append(s)
    return sims


# ---- CPU oracle baseline -----------------------------------------------------

def _oracle_worker(args):
    name, idx, steps = args
    os.environ["OMP_NUM_THREADS"] = "1"     # one thread per simulation process
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    cfg, parts = workload_cases(name)[idx]
    s = O.OracleSim(**cfg)
    for p in parts:
        s.add_particle(**p)
    s.step(1)                       # setup and first step outside the clock
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    return cfg["nx"] * cfg["ny"] * steps, dt


def cpu_baseline(steps_per_sim, name="sweep72", nsims=12):
    """The oracle as it stands (single-threaded C, FP64), one process per
    simulation of an evenly spaced sample of the workload's simulations (at
    most nsims), started with spawn; the rate is the sample's node updates
    over the slowest process's time."""
    from oracle import oracle as O
    O.build()
    total = len(workload_cases(name))
    nsims = min(nsims, total)
    cores = min(nsims, os.cpu_count() or 1)
    pick = [round(i * total / nsims) for i in range(nsims)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(name, i, steps_per_sim) for i in pick])
    wall = time.perf_counter() - t0
    updates = sum(r[0] for r in res)
    busy = max(r[1] for r in res) if cores >= nsims else sum(r[1] for r in res) / cores
    return {"value": updates / busy / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{nsims} of the {total} sims (every {total // nsims}th) x "
                      f"{steps_per_sim} steps, {cores} processes (wall {wall:.1f} s incl. setup)"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on a sample of the workload (12 of
    the 72 simulations, one worker process each), K timed steps or as many as
    fit in a few minutes."""
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    # bounded sample: cap the oracle work so that K steps end within minutes
    per_step_s = 0.06               # the largest sim (1024 x 256) per oracle step
    cap = max(1, int(150.0 / per_step_s))
    k_run = min(args.steps, cap)
    base = cpu_baseline(k_run + args.warmup * 0, args.workload)
    nodes = sum(c["nx"] * c["ny"] for c, _ in workload_cases(args.workload))
    line = {
        "metric": "aggregate MLUPS + % HBM roofline (FP32 vs FP16-storage), p50/p99 sim latency",
        "impl": "reference", "value": base["value"], "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": nodes / (base["value"] * 1e6) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOADS[args.workload][0],
                                        "storage": "f64 (oracle)"},
        "cpu_baseline": base,
        "e2e": {"value": base["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    if k_run < args.steps:
        line["cpu_baseline"]["sample"] += f"; {k_run} of {args.steps} steps timed"
    print(json.dumps(line))
    return 0


# ---- GPU arm -------------------------------------------------------------------

def max_over_ranks(x, device):
    """The largest x over the ranks of the default process group (x itself
    without one): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(world, nodes, steps, ms):
    """Whole-job rate: every rank updates `nodes` nodes per step (replicas),
    all ranks within the slowest rank's `ms`."""
    return world * nodes * steps / (ms * 1e-3) / 1e6


SAMPLE_GRAPHS = 16        # graph slots of the kernel-time sampler (lbib_batch_set_timing)
MIN_IN_REGION = 8         # in-region samples needed before they alone give the roofline
E2E_MIN_STEPS = 2048      # horizon of the end-to-end leg (a simulation request's length)


def bulk_timing(batch, kt_region):
    """Kernel times for the roofline: the samples taken inside the timed
    region (CUDA events around the kernels of one step per graph replay, and
    of the middle step of a call's steps outside a graph) when there are at
    least MIN_IN_REGION, else a sampled run of SAMPLE_GRAPHS graphs of 32
    steps right after the timed region, on the same batch and stream."""
    if kt_region["lattice_n"] >= MIN_IN_REGION:
        return kt_region, f"in the timed region ({kt_region['lattice_n']} sampled steps)"
    batch.step(32 * SAMPLE_GRAPHS)
    kt = batch.kernel_times()
    return kt, (f"sampled run of {32 * SAMPLE_GRAPHS} steps after the timed region "
                f"({kt['lattice_n']} sampled steps; {kt_region['lattice_n']} in the region)")


def storage_leg(lbib, W, storage, stream, alloc, steps, warmup, peak, rounding="stochastic",
                name="sweep72"):
    """The same workload with another storage format: step time, MLUPS and
    the bulk lattice pass against the HBM roofline at its bytes per update."""
    import torch
    sims = build_workload(lbib, W, storage, stream.cuda_stream, alloc, rounding, name)
    nodes = sum(s.nx * s.ny for s in sims)
    b = lbib.Batch(sims)
    b.step(2)
    variant, _ = b.autotune(20)
    b.set_timing(SAMPLE_GRAPHS)
    b.step(warmup)
    torch.cuda.synchronize()
    b.kernel_times()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kt, source = bulk_timing(b, b.kernel_times())
    pn = b.pass_nodes()
    b.synchronize()
    walls = wall_report(b, name, 2 + warmup + steps +
                        (32 * SAMPLE_GRAPHS if source.startswith("sampled run") else 0))
    bpu = BYTES_PER_UPDATE[storage]
    value = nodes * steps / (ms * 1e-3) / 1e6
    ach = pn["bulk"] * bpu / (kt["lattice_ms"] * 1e-3) / 1e9 if kt["lattice_ms"] > 0 else None
    b.close()
    for s in sims:
        s.close()
    return {"storage": storage, "rounding": rounding, "value": value, "unit": "MLUPS",
            "steps": steps, "ms_per_step": ms / steps, "bytes_per_update": bpu,
            "hbm_roofline_frac_of_step": value * 1e6 * bpu / (peak * 1e9),
            "lattice_kernel_ms": kt["lattice_ms"], "particle_kernel_ms": kt["particle_ms"],
            "near_kernel_ms": kt["near_ms"], "lattice_variant": variant,
            "kernel_timing": source, "bulk_le_step": kt["lattice_ms"] <= ms / steps,
            "roofline_achieved_gbs": ach, "roofline_frac": ach / peak if ach else None,
            "walls": walls}


def serving_leg(lbib, W, n_requests, alloc, quantum):
    """The serving loop on the first n_requests of the request trace (Poisson
    arrivals at 20/s, lattices 256x64 .. 2048x512, 1-4 particles, FP32 or
    FP16, 5k-50k steps) on the wall clock: p50 / p99 latency from arrival to
    result, served and offered update rates."""
    import torch
    from paper_1808_01448_gb300 import serve
    trace = W.serving_trace(n_requests)
    streams = {"f32": torch.cuda.Stream(), "f16": torch.cuda.Stream()}
    eng = serve.LbibEngine(lbib, {k: v.cuda_stream for k, v in streams.items()}, alloc)
    srv = serve.Server(eng, budget_bytes=150 << 30, quantum=quantum)
    t0 = time.perf_counter()
    res = srv.run(trace, t0=t0)
    wall = time.perf_counter() - t0
    eng.close()
    p50, p99 = serve.latency_stats(res)
    total = sum(r["steps"] * r["config"]["nx"] * r["config"]["ny"] for r in trace)
    return {"requests": len(res), "p50_s": p50, "p99_s": p99, "wall_s": wall,
            "served_mlups": srv.updates / wall / 1e6,
            "offered_mlups": total / trace[-1]["arrival_s"] / 1e6,
            "arrival_window_s": trace[-1]["arrival_s"], "rebuilds": srv.rebuilds,
            "rounds": srv.rounds, "quantum": quantum, "budget_gb": 150,
            "wall_s_in": {k: round(v, 3) for k, v in srv.time_in.items()},
            "admitted_in_place": srv.admitted_in_place,
            "trace": f"first {n_requests} requests of the 20/s Poisson trace (PCG64 seed 5)"}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1808_01448_gb300 import lbib
    from paper_1808_01448_gb300 import workloads as W

    rank, world = env_int("RANK", 0), env_int("WORLD_SIZE", 1)
    local = env_int("LOCAL_RANK", 0)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    # the oracle pool is spawned before any GPU work
    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(args.cpu_steps, args.workload)
    lbib.lib()
    stream = torch.cuda.Stream()
    alloc = lbib.torch_allocator()
    sims = build_workload(lbib, W, args.storage, stream.cuda_stream, alloc, name=args.workload)
    nodes = sum(s.nx * s.ny for s in sims)
    batch = lbib.Batch(sims)
    # pick the lattice-pass kernel variant on this batch (timing runs only)
    batch.step(2)
    variant, variant_ms = batch.autotune(20)
    if args.variant is not None:        # fixed choice (profiling runs)
        variant = args.variant
        batch.set_variant(variant)
    batch.set_timing(SAMPLE_GRAPHS)
    batch.step(args.warmup)
    torch.cuda.synchronize()
    batch.kernel_times()            # drop samples taken during warm-up

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    batch.step(args.steps)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    kt, kt_source = bulk_timing(batch, batch.kernel_times())
    pn = batch.pass_nodes()
    for s in sims:
        s.synchronize()             # raises on a device-side error
    walls = wall_report(batch, args.workload,
                        2 + args.warmup + args.steps +
                        (32 * SAMPLE_GRAPHS if kt_source.startswith("sampled run") else 0))
    ms = max_over_ranks(ms, "cuda")
    value = aggregate_mlups(world, nodes, args.steps, ms)

    # end to end through the C ABI with host buffers: fresh simulations, the
    # initial populations uploaded from pinned host memory, max(K, 2048) steps
    # (a request's length) in chunks of 128 with all particle states read back
    # to the host after each chunk
    e2e = None
    e2e_steps = max(args.steps, E2E_MIN_STEPS)
    if rank == 0 or world > 1:
        e2e_sims = build_workload(lbib, W, args.storage, stream.cuda_stream, alloc,
                                  name=args.workload)
        w9 = torch.tensor([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=torch.float64)
        f0 = {}                     # pinned initial populations, one per lattice shape
        for s in e2e_sims:
            if (s.ny, s.nx) not in f0:
                t = torch.empty((9, s.ny, s.nx), dtype=torch.float64).pin_memory()
                t.copy_(w9[:, None, None].expand(9, s.ny, s.nx))
                f0[(s.ny, s.nx)] = t.numpy()
        barrier()
        t0 = time.perf_counter()
        for s in e2e_sims:
            s.set_populations(f0[(s.ny, s.nx)])
        eb = lbib.Batch(e2e_sims)
        # every member's particle states after each chunk, one readback per
        # chunk, collected while the next chunk runs
        chunk, done, d2h, pending = 128, 0, 0, False
        while done < e2e_steps:
            n = min(chunk, e2e_steps - done)
            eb.step(n)
            done += n
            if pending:
                eb.particles()
                d2h += eb.last_d2h_bytes
            eb.read_particles_async()
            pending = True
        eb.particles()
        d2h += eb.last_d2h_bytes
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, "cuda")
        e2e = {"value": aggregate_mlups(world, nodes, e2e_steps, dt * 1e3), "unit": "MLUPS",
               "h2d_bytes_per_step": world * 9 * nodes * 8 / e2e_steps,
               "d2h_bytes_per_step": world * d2h / e2e_steps, "steps": e2e_steps,
               "includes": "simulation and batch set-up, initial populations uploaded from "
                           "pinned host memory, all particle states read back every 128 steps"}
        eb.close()
        for s in e2e_sims:
            s.close()

    peak, peak_kind = read_peaks()
    legs = {}
    if rank == 0 and args.storage == "f32" and args.storage_steps > 0:
        legs["fp16_storage"] = storage_leg(lbib, W, "f16", stream, alloc, args.storage_steps,
                                           args.warmup, peak, name=args.workload)
        legs["bf16_storage"] = storage_leg(lbib, W, "bf16", stream, alloc, args.storage_steps,
                                           args.warmup, peak, name=args.workload)
    if rank == 0 and args.serve_requests > 0:
        legs["latency"] = serving_leg(lbib, W, args.serve_requests, alloc, args.serve_quantum)

    if rank == 0:
        bpu = BYTES_PER_UPDATE[args.storage]
        l2_mib = torch.cuda.get_device_properties(local).L2_cache_size / 2**20
        lat_ms = kt["lattice_ms"]
        # algorithmic bytes of one bulk-pass launch: the nodes it updates
        achieved = pn["bulk"] * bpu / (lat_ms * 1e-3) / 1e9 if lat_ms > 0 else None
        per_step = 3 if kt["near_n"] else 2
        launches = per_step * args.steps + (1 if args.steps % 2 else 0)
        line = {
            "metric": "aggregate MLUPS + % HBM roofline (FP32 vs FP16-storage), p50/p99 sim latency",
            "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][0],
                       "lattices": WORKLOADS[args.workload][1], "nodes": nodes,
                       "sims": len(sims),
                       "storage": args.storage,
                       "l2": (f"inputs larger than L2, no flush: {nodes * bpu / 1e6:.0f} MB of "
                              f"populations (two buffers) vs {l2_mib:.0f} MiB L2"
                              if nodes * bpu > l2_mib * 2**20 else
                              f"inputs smaller than L2 ({nodes * bpu / 1e6:.0f} MB of populations "
                              f"vs {l2_mib:.0f} MiB), steps back to back without a flush: "
                              f"not a cold-cache timing"),
                       "parallelism": f"replicas x{world}"},
            "hbm_roofline_frac_of_step": value * 1e6 * bpu / (peak * 1e9) / world,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if achieved else None,
                         "traffic": ncu_traffic(args.storage), "peak_source": peak_kind,
                         "kernel": "lattice_kernel", "bytes_per_update": bpu,
                         "lattice_kernel_ms": lat_ms, "particle_kernel_ms": kt["particle_ms"],
                         "near_kernel_ms": kt["near_ms"], "nodes_per_launch": pn["bulk"],
                         "lattice_variant": variant,
                         "variant_ms": [round(x, 5) for x in variant_ms],
                         "alone_ms": round(variant_ms[variant], 5),
                         "samples": kt["lattice_n"], "timing": kt_source,
                         "bulk_le_step": lat_ms <= ms / args.steps},
            "walls": walls, "clocks": clk, "e2e": e2e, "gpu_launches": launches,
            "cpu_baseline": base,
        }
        line.update(legs)
        print(json.dumps(line))
    batch.close()
    for s in sims:
        s.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=64)
    ap.add_argument("--impl", default="lbib", choices=["lbib", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16", "f64"])
    ap.add_argument("--cpu-steps", type=int, default=300)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--storage-steps", type=int, default=2000,
                    help="steps of the FP16 / BF16 storage legs (0: skip)")
    ap.add_argument("--serve-requests", type=int, default=60,
                    help="requests of the serving leg (0: skip)")
    ap.add_argument("--serve-quantum", type=int, default=1000)
    ap.add_argument("--workload", default="sweep72", choices=sorted(WORKLOADS),
                    help="sweep72: the 72-channel design sweep (inputs larger than L2); "
                         "ellipse6: six 1024x256 channels (inputs fit in L2)")
    ap.add_argument("--variant", type=int, default=None,
                    help="lattice-pass kernel variant instead of the autotuner's choice")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
