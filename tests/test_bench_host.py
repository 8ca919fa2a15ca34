"""CPU checks of bench.py's host logic: the reference (oracle) arm's JSON
line (one oracle process per host core), and the whole-job aggregation
across ranks (max of the ranks' times, sum of their work) run as two gloo
processes."""
import json
import os
import socket
import subprocess
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--size", "48",
                        "--sample", "24", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["value"] > 0
    cores = len(os.sched_getaffinity(0))
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == cores
    assert d["cpu_baseline"]["nproc"] == cores and d["cpu_baseline"]["cpu_model"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench

    def reduce_max(v):
        t = torch.tensor([v], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    t, gbs = bench.aggregate_ranks(local_ms, world, 1000, reduce_max)
    out[rank] = (t, gbs)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregation_over_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        t, gbs = out[rank]
        assert t == 15.0  # the slowest rank's time
        assert abs(gbs - world * 4.0 * 1000 / 15e-3 / 1e9) < 1e-12
