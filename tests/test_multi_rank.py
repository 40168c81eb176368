"""The bench's multi-GPU path is replicas: per-rank timing is combined as the max over ranks and
the work as the sum.  Checked here with world_size-2 gloo process groups on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    w, r, l = bench.dist_env()
    t_max = bench.allreduce(10.0 + rank, "max", world)   # each rank's timed milliseconds
    work = bench.allreduce(100.0 * (rank + 1), "sum", world)  # each rank's voxel-iterations
    bench.barrier(world)
    q.put((rank, w, r, l, t_max, work))
    dist.destroy_process_group()


def test_replica_timing_reduction_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, r, l, t_max, work in out:
        assert (w, r, l) == (2, rank, rank)
        assert t_max == 11.0      # the slowest rank sets the time
        assert work == 300.0      # whole-job work is the sum over ranks


def test_bench_launcher_starts_its_own_ranks():
    # bench.py --gpus 2 without an external launcher starts two ranks itself (gloo on the CPU here):
    # ranks 0 and 1 on devices cuda:0 and cuda:1, one JSON line from rank 0 with the max of the
    # ranks' times and the sum of their work, and n_gpus = the ranks that ran
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_PORT")}
    env["ELAS_BENCH_BACKEND"] = "gloo"
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--launcher-selftest"],
                       capture_output=True, text=True, timeout=300, env=env, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    assert out["n_gpus"] == 2
    assert [(q["rank"], q["local_rank"], q["device"], q["world"]) for q in out["ranks"]] == [
        (0, 0, "cuda:0", 2), (1, 1, "cuda:1", 2)]
    assert out["t_max_ms"] == 11.0 and out["work"] == 300.0
