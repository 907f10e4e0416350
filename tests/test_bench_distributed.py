"""The multi-process form of the benchmark on CPU (gloo, two ranks): every
rank reconstructs its own batch, the step time is the maximum over ranks, the
value counts the events of all ranks, and the reference arm runs on rank 0
only.  No GPU: the reduction and the rank handling are host logic."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, ws: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_2207_03936_gb300 import synth
    ws_env, rank_env, local_env = bench.dist_env()
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms_local = 10.0 + 2.5 * rank            # the last rank is the slowest
        ms_max, value = bench.job_throughput(ms_local, 1000, ws_env, dist)
        ev = synth.make_events(1, 3, seed=rank_env, workers=1)   # the seed the bench gives each rank
        q.put(dict(rank=rank, env=(ws_env, rank_env, local_env), ms_max=ms_max, value=value,
                   first_x=float(ev.x[0])))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort(key=lambda d: d["rank"])
    assert [d["env"] for d in got] == [(2, 0, 0), (2, 1, 1)]
    for d in got:
        assert d["ms_max"] == 12.5                      # max over ranks, on every rank
        assert np.isclose(d["value"], 2 * 1000 / 0.0125)  # events of both ranks / slowest step
    assert got[0]["first_x"] != got[1]["first_x"]        # each rank has its own events


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    ms_max, value = bench.job_throughput(20.0, 500, 1)
    assert ms_max == 20.0 and np.isclose(value, 500 / 0.02)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--events", "50", "--cpu-seconds", "0.1"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--events", "50", "--cpu-seconds", "0.1"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
