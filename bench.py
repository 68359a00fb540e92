"""Benchmark: RSOS site-update attempts/s on one GB300 (per GPU of a node).

One step is one whole multisurface job through the C ABI: flat init, 10^4
double-tiling sweeps of an L = 4096 periodic lattice with N = 1 and 64
surfaces in uint64 words (8x8 tiles, seed = 0 + rank), exact sum h / sum h^2
at 40 log-spaced times, and the read-back of the W^2 series.  value =
L^2 * S * sweeps / time (expected attempts, one sweep = 1 MCS).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (the reference arm of this project:
there is no reference code, only the paper) on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RSOS site-update attempts/s on 1 GB300 (plain vs batched); % HBM roofline"
WORKLOAD = dict(workload="ms-n1: L=4096 periodic, N=1, 64 surfaces bit-sliced in uint64 words, 8x8 DT tiles, "
                         "flat start, 1e4 sweeps, W^2 per surface at 40 log-spaced times",
                L=4096, N=1, surfaces=64, tile=8, tiling=0, sweeps=10000, measurements=40)
# The (+1) tilings of the decomposition check (section III.C) on the paper's
# largest lattice, which no regular tile divides (9605 = 5 x 17 x 113).
WORKLOAD_IRREGULAR = dict(workload="ms-irregular: L=9605 periodic, N=1, 64 surfaces bit-sliced in uint64 words, "
                                   "6(+1)x10(+1) DT tiles, flat start, 2000 sweeps, W^2 per surface at 30 "
                                   "log-spaced times",
                          L=9605, N=1, surfaces=64, tile=(6, 10), tiling=1, sweeps=2000, measurements=30)
CSRC = "paper_1605_02620_gb300/csrc/"
KERNELS = {
    0: dict(name="rsos::persistent_kernel<1, uint64_t, 4>", launches_per_sweep=None,
            profile="persistent_kernel_L4096_N1_S64.md",
            sources=["rsos_device.cuh", "rsos_persist.cuh", "rsos_sched.cuh", "rsos_logic.cuh", "philox.cuh",
                     "rsos_persist_launch.cuh"]),
    1: dict(name="rsos::general_phase_kernel<1, uint64_t>", launches_per_sweep=4,
            profile="general_phase_kernel_L9605_N1_S64.md",
            sources=["rsos_device.cuh", "rsos_general.cu", "rsos_general.cuh", "rsos_logic.cuh", "philox.cuh"]),
}


def kernel_hash(tiling: int = 0) -> str:
    h = hashlib.sha256()
    for rel in KERNELS[tiling]["sources"]:
        with open(os.path.join(ROOT, CSRC + rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(tiling: int = 0):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    try:
        text = open(os.path.join(ROOT, "profiles", KERNELS[tiling]["profile"])).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_hash(tiling):
        return None
    return float(t.group(1))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "of measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "of fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[3 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_setup(n_gpus: int):
    """Ranks from the torchrun environment; one process group for the
    timing reductions (NCCL with GPUs, gloo on a host without).  A rank that
    dies or never arrives ends the others' next collective with an error after
    RSOS_DIST_TIMEOUT_S seconds (default 600) instead of a hang."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import datetime

        import torch
        import torch.distributed as dist
        timeout = datetime.timedelta(seconds=float(os.environ.get("RSOS_DIST_TIMEOUT_S", "600")))
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", timeout=timeout)
        else:
            dist.init_process_group("gloo", timeout=timeout)
    return world, rank, local


def dist_max(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(attempts_per_rank_step: float, world: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: every rank ran ``steps`` jobs of the same size;
    the slowest rank's time bounds the job."""
    return attempts_per_rank_step * world * steps / (max_ms / 1e3)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_gpu(args):
    import torch

    import paper_1605_02620_gb300 as R
    from paper_1605_02620_gb300.inputs import log_schedule

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    W = WORKLOAD
    L, S, sweeps = W["L"], W["surfaces"], W["sweeps"]
    times = log_schedule(sweeps, W["measurements"])
    seed = rank
    params = R.rsos_params(L=L, N=W["N"], surfaces=S, tile=W["tile"], seed=seed,
                           series_capacity=len(times) + 1, tiling=W["tiling"])
    nbytes = R.rsos_required_bytes(params)
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = (buf.data_ptr() + 255) // 256 * 256

    launches = [0]

    def one_job(device_timed=True):
        h = R.rsos_init(params, dev_buf=base, dev_bytes=nbytes, stream=stream)
        R.rsos_schedule(h, times)
        R.rsos_sweep(h, sweeps, stream=stream)
        ts, s1, s2, w2 = R.rsos_read_series(h, S, len(times) + 1, stream=stream)
        launches[0] = R.rsos_launches(h)
        R.rsos_free(h)
        return ts, w2

    for _ in range(args.warmup):
        one_job()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        ts, w2 = one_job()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    dev_ms = ev0.elapsed_time(ev1)
    dev_ms = dist_max(dev_ms, world)
    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "ms_per_step": dev_ms / args.steps, "sweeps": sweeps}), flush=True)
        return

    # Dominant kernel, timed alone on the same stream: one persistent launch
    # of n_kernel_sweeps sweeps (no measurement inside), or, on a (+1)
    # tiling, the 4 n_kernel_sweeps phase launches of as many sweeps.
    h = R.rsos_init(params, dev_buf=base, dev_bytes=nbytes, stream=stream)
    R.rsos_sweep(h, 50, stream=stream)
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_kernel_sweeps = 200
    k0.record(stream)
    R.rsos_sweep(h, n_kernel_sweeps, stream=stream)
    k1.record(stream)
    torch.cuda.synchronize()
    R.rsos_free(h)
    launch_ms = k0.elapsed_time(k1)

    # End to end through the public API with host buffers: the library
    # allocates device memory, runs, and the series is copied to host arrays.
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 2))
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        p2 = R.rsos_params(L=L, N=W["N"], surfaces=S, tile=W["tile"], seed=seed, series_capacity=len(times) + 1,
                           tiling=W["tiling"])
        h = R.rsos_init(p2, stream=stream)
        R.rsos_schedule(h, times)
        R.rsos_sweep(h, sweeps, stream=stream)
        R.rsos_read_series(h, S, len(times) + 1, stream=stream)
        R.rsos_free(h)
    torch.cuda.synchronize()
    e2e_s = dist_max(time.perf_counter() - t0, world)

    attempts = float(L) * L * S * sweeps
    value = aggregate_rate(attempts, world, args.steps, dev_ms)
    e2e_value = aggregate_rate(attempts, world, e2e_steps, e2e_s * 1e3)
    peaks, peak_src = measured_peaks()
    K = KERNELS[W["tiling"]]
    # launches in the kernel-timing region: one persistent launch, or four
    # phase launches per sweep
    n_launch = K["launches_per_sweep"] * n_kernel_sweeps if K["launches_per_sweep"] else 1
    alg_bytes = 2.0 * (rsos_bits(W["N"]) / 8.0) * L * L * S * n_kernel_sweeps / n_launch  # per launch
    per_launch_ms = launch_ms / n_launch
    achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9
    launches_per_job = launches[0]
    if rank != 0:
        return
    cpu = cpu_baseline(L, W["N"], W["tile"], seed, tiling=W["tiling"]) if world == 1 else None
    # Integer-pipe side of the roofline: measured lop3 / mad.lo lane rates and
    # Philox blocks/s.  A 64-lane selection draws 1/8 site block and 2/4 mask
    # blocks; each lane sees two selections per expected attempt.
    philox_per_attempt = (1.0 / 8 + 2.0 / 4) * 2.0 / 64
    int_peaks = {"lop3_lane_ops_per_s": R.rsos_peak_int(0, 4096, stream),
                 "imad_lane_ops_per_s": R.rsos_peak_int(1, 4096, stream),
                 "philox_blocks_per_s": R.rsos_peak_int(2, 512, stream)}
    int_peaks["philox_bound_attempts_per_s"] = int_peaks["philox_blocks_per_s"] / philox_per_attempt
    lanes_note = f"inputs larger than L2 ({L * L * S * rsos_bits(W['N']) / 8 / 2 ** 20:.0f} MiB lattice per job)"
    line = {
        "metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64 (bit-sliced int)", "data": "synthetic",
        "config": dict(W, parallelism=f"replicas{world}", l2=lanes_note, seed=seed),
        "e2e": {"value": e2e_value, "unit": "attempts/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": (len(times)) * S * 4 * 8 + 8},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": profiled_traffic(W["tiling"]),
                     "kernel": K["name"], "launch_ms": per_launch_ms,
                     "sweeps_per_launch": n_kernel_sweeps / n_launch,
                     "algorithmic_bytes_per_launch": alg_bytes, "peak_source": peak_src},
        "cpu_baseline": cpu,
        "int_peaks": int_peaks,
        "clocks": clk,
        "gpu_launches": launches_per_job * args.steps,
        "w2_final_mean": float(sum(w2[-1]) / len(w2[-1])),
    }
    print(json.dumps(line), flush=True)


def rsos_bits(N: int) -> int:
    return 2 if N <= 1 else (3 if N <= 3 else 4)


def _edges(T):
    return (T, T) if not isinstance(T, (tuple, list)) else tuple(T)


def cpu_baseline(L, N, T, seed, target_s: float = 12.0, tiling: int = 0):
    """The oracle, as it stands, on the host cores: one DT sweep of the
    workload's lattice for as many lanes as there are cores (one lane per
    thread), repeated until about ``target_s`` seconds of CPU work."""
    import oracle as O
    cores = os.cpu_count() or 1
    Tx, Ty = _edges(T)
    p = O.Params(L=L, N=N, Tx=Tx, Ty=Ty, seed=seed, tiling=tiling)
    lanes = list(range(cores))
    h = O.flat(L, cores)
    done, t0 = 0, time.perf_counter()
    while True:
        O.sweeps(p, h, lanes, done, 1, threads=cores)
        done += 1
        el = time.perf_counter() - t0
        if el > target_s or done >= 8:
            break
    value = float(L) * L * cores * done / el
    return {"value": value, "unit": "attempts/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} DT sweep(s) of L={L}, N={N}, {cores} lanes, {cores} threads, from the flat start"}


def run_batched(args):
    """Batched workload: 256 independent jobs (L uniform in {256..4096}, N in
    {1, 2}, 64 surfaces, t_max log-uniform in [1e3, 1e4] sweeps, seeds =
    job index), one multi-job persistent launch per class, captured in a CUDA
    graph; each job's width is measured exactly at its t_max.  One step = the
    whole batch."""
    import torch

    import paper_1605_02620_gb300 as R
    from paper_1605_02620_gb300.inputs import batched_jobs

    scale = args.batch_scale
    jobs = batched_jobs()
    # execution geometry per (L, N) from the autotuner (untimed set-up; the
    # results do not depend on it)
    geometry = {}
    for L, N in sorted({(j["L"], j["N"]) for j in jobs}):
        tuned, _ = R.rsos_autotune(R.rsos_params(L=L, N=N, surfaces=64, tile=8), sweeps=10)
        geometry[(L, N)] = (tuned.words_per_thread, tuned.tiles_per_lane, tuned.phase_lag)
    params = [R.rsos_params(L=j["L"], N=j["N"], surfaces=j["surfaces"], tile=8, seed=j["seed"], series_capacity=2,
                            **dict(zip(("words_per_thread", "tiles_per_lane", "phase_lag"),
                                       geometry[(j["L"], j["N"])])))
              for j in jobs]
    tmax = [max(1, j["t_max"] // scale) for j in jobs]
    attempts = float(sum(j["L"] * j["L"] * j["surfaces"] * t for j, t in zip(jobs, tmax)))
    stream = torch.cuda.Stream()

    def one_batch(tm=None):
        b = R.rsos_batch_create(params, tm or tmax)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        R.rsos_batch_run(b, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        done = set()
        while len(done) < len(jobs):
            _, ids = R.rsos_batch_poll(b)
            done |= set(ids)
        w2 = [float(R.rsos_read_series(R.rsos_batch_job(b, k), jobs[k]["surfaces"], 2)[3][-1].mean())
              for k in range(0, len(jobs), 64)]
        R.rsos_batch_free(b)
        return ev0.elapsed_time(ev1), w2

    # warm-up: the same batch with t_max / 100 (compiles plans, warms clocks)
    warm_tmax = [max(1, t // 100) for t in tmax]
    for _ in range(args.warmup):
        one_batch(warm_tmax)
    clocks = ClockSampler(0)
    clocks.start()
    total_ms = 0.0
    for _ in range(args.steps):
        ms, w2 = one_batch()
        total_ms += ms
    clk = clocks.stop()
    value = attempts * args.steps / (total_ms / 1e3)

    # The same jobs one at a time: each (L, N) of the mix timed alone (one
    # job of 64 surfaces, device time of ~50 ms of sweeps after 20 warm-up
    # sweeps), then every job charged at its own rate.
    rates = {}
    for L, N in sorted({(j["L"], j["N"]) for j in jobs}):
        wpt, tpl, lag = geometry[(L, N)]
        h = R.rsos_init(R.rsos_params(L=L, N=N, surfaces=64, tile=8, seed=0, series_capacity=2,
                                      words_per_thread=wpt, tiles_per_lane=tpl, phase_lag=lag), stream=stream)
        R.rsos_sweep(h, 20, stream=stream)
        n = max(20, int(5e10 / (L * L * 64 * (1.0 if N == 1 else 2.0)) / 5))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        R.rsos_sweep(h, n, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        rates[(L, N)] = L * L * 64 * n / (e0.elapsed_time(e1) / 1e3)
        R.rsos_free(h)
    alone_s = sum(j["L"] * j["L"] * j["surfaces"] * t / rates[(j["L"], j["N"])] for j, t in zip(jobs, tmax))
    plain_equiv = attempts / alone_s
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64/u32 (bit-sliced int)", "data": "synthetic",
        "plain_equivalent": {"value": plain_equiv, "unit": "attempts/s", "ratio": value / plain_equiv,
                             "how": "the same jobs run one at a time, each at its own (L, N) single-job rate "
                                    "with the same autotuned geometry",
                             "rates": {f"L{L}_N{N}": r for (L, N), r in rates.items()}},
        "config": {"workload": f"batched: 256 jobs, L in {{256..4096}}, N in {{1,2}}, 64 surfaces, t_max in "
                               f"[1e3,1e4]/{scale} sweeps, PCG64 seed 2016; one multi-job persistent launch per class "
                               "in a CUDA graph; execution geometry per (L, N) from rsos_autotune",
                   "jobs": len(jobs), "attempts_per_step": attempts,
                   "geometry": {f"L{L}_N{N}": list(g) for (L, N), g in geometry.items()},
                   "l2": "inputs larger than L2"},
        "clocks": clk, "w2_sample": w2,
    }), flush=True)


def run_served(args):
    """Served workload: a Poisson stream of requests (L = 2^e, e in 8..13, N in
    1..4, 64 surfaces, t_max log-uniform in [1e2, 1e4] sweeps, PCG64 seed
    2017) admitted under an HBM budget by the continuous-batching server.
    --serve-jobs / --serve-scale (t_max divisor) / --serve-rate (arrivals per
    second) bound the run; the JSON line states them."""
    import torch

    from paper_1605_02620_gb300.inputs import served_jobs
    from paper_1605_02620_gb300.serve import Request, Server

    jobs = served_jobs(n_jobs=args.serve_jobs, rate=args.serve_rate)
    reqs = [Request(L=j["L"], N=j["N"], t_max=max(1, j["t_max"] // args.serve_scale), seed=j["seed"],
                    surfaces=j["surfaces"], arrival=j["arrival"], rid=k) for k, j in enumerate(jobs)]
    stream = torch.cuda.Stream()
    warm = [Request(L=256, N=n, t_max=20, seed=k, surfaces=64, arrival=0.0, rid=k) for k, n in enumerate((1, 2, 3, 4))]
    # warm-up: also tunes every job shape of the stream (cached; untimed)
    shapes = sorted({(r.L, r.N, r.surfaces) for r in reqs})
    Server(hbm_budget=args.serve_budget, stream=stream, tune=True).run(
        warm + [Request(L=L, N=N, t_max=1, seed=0, surfaces=S, arrival=0.0, rid=-1 - k)
                for k, (L, N, S) in enumerate(shapes)])
    clocks = ClockSampler(0)
    clocks.start()
    rep = Server(hbm_budget=args.serve_budget, epoch_s=args.serve_epoch, stream=stream, tune=True).run(reqs)
    clk = clocks.stop()
    s = rep.summary()
    print(json.dumps({
        "metric": METRIC, "value": s["attempts_per_s"], "unit": "attempts/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": rep.wall_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64/u32 (bit-sliced int)", "data": "synthetic",
        "config": {"workload": f"served: {len(reqs)} Poisson requests at {args.serve_rate}/s, L=2^(8..13), N in 1..4, "
                               f"64 surfaces, t_max in [1e2,1e4]/{args.serve_scale} sweeps, PCG64 seed 2017",
                   "hbm_budget": args.serve_budget, "epoch_s": args.serve_epoch,
                   "geometry": "per job shape from rsos_autotune (tuned in the warm-up)"},
        "serve": s, "clocks": clk,
    }), flush=True)


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    W = WORKLOAD
    cores = os.cpu_count() or 1
    L = W["L"]
    Tx, Ty = _edges(W["tile"])
    p = O.Params(L=L, N=W["N"], Tx=Tx, Ty=Ty, seed=0, tiling=W["tiling"])
    lanes = list(range(cores))
    h = O.flat(L, cores)
    for k in range(args.warmup):
        O.sweeps(p, h, lanes, k, 1, threads=cores)
    t0 = time.perf_counter()
    for k in range(args.steps):
        O.sweeps(p, h, lanes, args.warmup + k, 1, threads=cores)
    el = time.perf_counter() - t0
    value = float(L) * L * cores * args.steps / el
    sample = f"{args.steps} DT sweep(s) of L={L}, N={W['N']}, {cores} lanes, {cores} threads"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": dict(W, parallelism="host threads", note="each step is one sweep of cores lanes (bounded sample)"),
        "cpu_baseline": {"value": value, "unit": "attempts/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--sweeps", type=int, default=WORKLOAD["sweeps"],
                    help="sweeps per job (reduced values only for profiling captures)")
    ap.add_argument("--measurements", type=int, default=WORKLOAD["measurements"],
                    help="measurement times per job (reduced values only for profiling captures)")
    ap.add_argument("--workload", default="ms-n1", choices=["ms-n1", "irregular", "batched", "served"])
    ap.add_argument("--batch-scale", type=int, default=1,
                    help="divide the batched jobs' t_max by this factor (profiling / quick checks)")
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-scale", type=int, default=1)
    ap.add_argument("--serve-budget", type=int, default=200 << 30)
    ap.add_argument("--serve-epoch", type=float, default=0.02)
    ap.add_argument("--quick", action="store_true",
                    help="profiling capture: timed steps only (no kernel timing, e2e or CPU baseline)")
    args = ap.parse_args()
    if args.workload == "irregular":
        WORKLOAD.clear()
        WORKLOAD.update(WORKLOAD_IRREGULAR)
        if "--sweeps" not in sys.argv:
            args.sweeps = WORKLOAD["sweeps"]
        if "--measurements" not in sys.argv:
            args.measurements = WORKLOAD["measurements"]
    if args.sweeps != WORKLOAD["sweeps"] or args.measurements != WORKLOAD["measurements"]:
        WORKLOAD["sweeps"] = args.sweeps
        WORKLOAD["measurements"] = max(2, min(args.measurements, args.sweeps))
        WORKLOAD["workload"] += (f" [reduced to {args.sweeps} sweeps, {WORKLOAD['measurements']} measurements"
                                 " for profiling]")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
