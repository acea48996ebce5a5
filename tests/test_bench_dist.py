"""The multi-rank logic of bench.py on CPU: two gloo ranks (the replicas
layout the GPU bench uses under torchrun, where every rank renders its own
walk and only the timing is reduced), and the reference arm under torchrun,
where rank 0 alone runs and prints."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import scenegen
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = bench.max_over_ranks(10.0 + rank, ws, device="cpu")
    heading, start = bench.rank_walk(scenegen.CONFIGS["city"], rank)
    cam = scenegen.trajectory("city", 5, heading, start)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, [float(x) for x in cam["pos"]]))


def test_two_gloo_ranks_reduce_time_and_walk_apart():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [11.0, 11.0]          # every rank sees the slowest rank's time
    assert abs((res[1][2][1] - res[0][2][1]) - 40.0) < 1e-3  # rank 1 walks the street 40 m over
    assert res[1][2][0] == res[0][2][0]


def test_reference_arm_under_torchrun_rank0_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--config", "tiny", "--gpus", "2", "--steps", "2", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
