"""The multi-rank host logic of bench.py on CPU: two gloo ranks (one process
each) agree on the slowest rank's time and on the whole-job rate, and the
reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(times[rank], "cpu")
    out[rank] = (ms, bench.aggregate_mlups(world, 1000, 50, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world, port = 2, _free_port()
    times = [3.5, 4.25]
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == max(times)
    assert value == pytest.approx(world * 1000 * 50 / (max(times) * 1e-3) / 1e6)


def test_single_process_reduction_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, "cpu") == 1.25


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "3", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_wall_report_takes_each_channels_height():
    """y_min over H per particle with H = ny - 1 (Zou-He wall rows) or ny
    (bounce-back), the crossing count and the bonded count."""
    sys.path.insert(0, ROOT)
    import bench
    cases = bench.workload_cases("ellipse6")

    class FakeBatch:
        def particles(self):
            rows = []
            for k, (c, _) in enumerate(cases):
                rows.append([{"gap_bottom": (k - 1) * 0.01 * (c["ny"] - 1), "n_bonded": k % 2}])
            return rows

    r = bench.wall_report(FakeBatch(), "ellipse6", 100)
    assert r["particles"] == len(cases)
    assert r["y_min_over_h"] == pytest.approx(-0.01)
    assert r["crossed"] == 2              # gaps -0.01 H and 0
    assert r["bonded_particles"] == len(cases) // 2
    assert r["after_steps"] == 100
