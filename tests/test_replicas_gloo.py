"""The multi-GPU path of bench.py is "replicas only": every rank runs its own
independent job (seed = rank) and the ranks meet only to agree on the
slowest rank's time.  These tests run that host logic as two gloo ranks on
the CPU: the max-over-ranks reduction, the barrier, the aggregate rate, and
the reference arm launched by torchrun (rank 0 alone prints one line), and
a rank that dies before the barrier: the survivor's collective ends with an
error within the process-group timeout instead of hanging."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_setup(world)
    worst = bench.dist_max(100.0 + 50.0 * r, w)  # rank 1 is the slow one
    bench.barrier(w)
    rate = bench.aggregate_rate(1e9, w, 3, worst)
    dist.destroy_process_group()
    q.put((r, w, worst, rate))


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, worst, rate in out:
        assert w == 2 and worst == 150.0
        # two ranks x 3 jobs of 1e9 attempts in the slowest rank's 150 ms
        assert rate == pytest.approx(2 * 3 * 1e9 / 0.150)


def test_reference_arm_under_torchrun_world_2():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def _rank_dies(rank: int, world: int, port: int, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="", RSOS_DIST_TIMEOUT_S="10")
    sys.path.insert(0, ROOT)
    import time

    import bench
    w, r, _ = bench.dist_setup(world)
    if r == 1:
        os._exit(3)  # simulated worker death between steps, nothing in flight
    t0 = time.perf_counter()
    try:
        bench.barrier(w)
        bench.dist_max(1.0, w)
        q.put(("no error", time.perf_counter() - t0))
    except Exception as e:  # the collective with a dead peer must fail
        q.put((type(e).__name__, time.perf_counter() - t0))


def test_dead_rank_ends_the_survivors_collective_with_an_error():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_dies, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    kind, waited = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert kind != "no error"
    assert waited < 60  # bounded by the 10 s process-group timeout (plus slack)
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0
