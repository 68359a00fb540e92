"""Benchmark: RSOS site-update attempts/s on one GB300 (per GPU of a node).

One step is one whole multisurface job through the C ABI: flat init, 10^4
double-tiling sweeps of an L = 4096 periodic lattice with N = 1 and 64
surfaces in uint64 words (8x8 tiles, seed = 0 + rank), exact sum h / sum h^2
at 40 log-spaced times, and the read-back of the W^2 series.  value =
L^2 * S * sweeps / time (expected attempts, one sweep = 1 MCS).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --workload {ms-n1,irregular,step-height,batched,served} [--N n]

--impl reference times the CPU oracle (the reference arm of this project:
there is no reference code, only the paper) on a bounded sample of the same
workload on the host cores.

The roofline of every line is the slower of two bounds computed from the
method's own work per expected attempt: the HBM bound (one read and one
write of B bits per site and surface per sweep) and the integer-pipe bound
(Philox blocks on the FMA pipe and 3-input logic on the ALU pipe, both at
the rates rsos_peak_int measures on this GPU); see int_bound().
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


def step_height_workload(N: int) -> dict:
    """The step-height runs (section II: growth at N = 1, 3, 5, 7 on the
    largest lattices): L = 32768 with 32 surfaces (8, 12 or 16 GiB of planes
    at N = 1, 2, 4), the timed prefix of 1e3 of the 1e5 sweeps."""
    return dict(workload=f"step-height: L=32768 periodic, N={N}, 32 surfaces bit-sliced in uint32 words, 8x8 DT "
                         "tiles, flat start, 1e3 sweeps (the timed prefix of 1e5), W^2 per surface at 20 "
                         "log-spaced times",
                L=32768, N=N, surfaces=32, tile=8, tiling=0, sweeps=1000, measurements=20)

CSRC = "paper_1605_02620_gb300/csrc/"
KERNELS = {
    "persistent": dict(launches_per_sweep=None,
                       sources=["rsos_device.cuh", "rsos_persist.cuh", "rsos_sched.cuh", "rsos_logic.cuh",
                                "philox.cuh", "rsos_persist_launch.cuh"]),
    "general": dict(launches_per_sweep=4,
                    sources=["rsos_device.cuh", "rsos_general.cu", "rsos_general.cuh", "rsos_logic.cuh",
                             "philox.cuh"]),
}
# committed ncu summary per workload (the profile whose DRAM bytes give roofline.traffic)
PROFILES = {"ms-n1": "persistent_kernel_L4096_N1_S64.md", "irregular": "general_phase_kernel_L9605_N1_S64.md",
            "step-height-1": "persistent_kernel_L32768_N1_S32.md", "step-height-2": "persistent_kernel_L32768_N2_S32.md",
            "step-height-4": "persistent_kernel_L32768_N4_S32.md"}


def lanes_per_thread(N: int, S: int) -> int:
    """Surfaces one thread of the sweep kernels updates per selection (32 or 64):
    the library's automatic choice of words per thread."""
    NW = (S + 31) // 32
    if NW % 2 != 0 or (rsos_bits(N) >= 3 and NW <= 32):
        return 32
    return 64


def int_bound(N: int, lanes: int, int_peaks: dict) -> dict:
    """Integer-pipe bound of the sweep from the method's work per expected
    attempt.  Each lane sees two selections per expected attempt (2a
    selections, half masks); a thread of `lanes` surfaces draws per selection
    1/8 Philox block for the site (eight 16-bit draws per block) and 1/4 block
    per 32-lane word for the masks.  Philox-4x32-10 is bound by its wide
    multiplies (FMA pipe): its time is blocks / the measured block rate.  The
    ALU pipe (3-input logic) runs Philox's two 3-way XORs per round (20 per
    block) and the bit-sliced Eq. 6 test and ripple increment, 8B - 1 per
    32-lane word per selection (y = x - N: 2B - 2; four neighbour
    comparisons: 4B; the mask AND: 2; increment: 2B - 1)."""
    B = rsos_bits(N)
    words = lanes / 32.0
    sel = 2.0 / lanes  # selections of a thread per lane-attempt
    blocks = sel * (1.0 / 8 + words / 4)
    alu = 20.0 * blocks + sel * words * (8 * B - 1)
    t_fma = blocks / int_peaks["philox_blocks_per_s"]
    t_alu = alu / int_peaks["lop3_lane_ops_per_s"]
    return {"attempts_per_s": 1.0 / max(t_fma, t_alu), "pipe": "fma (philox)" if t_fma > t_alu else "alu (lop3)",
            "philox_blocks_per_attempt": blocks, "alu_ops_per_attempt": alu, "lanes_per_thread": lanes}


def measure_int_peaks(R, stream) -> dict:
    return {"lop3_lane_ops_per_s": R.rsos_peak_int(0, 4096, stream),
            "imad_lane_ops_per_s": R.rsos_peak_int(1, 4096, stream),
            "philox_blocks_per_s": R.rsos_peak_int(2, 512, stream)}


def roofline_of(parts, seconds: float, peaks: dict, peak_src: str, int_peaks: dict, **extra) -> dict:
    """Roofline of work done in `seconds`: parts = [(attempts, N, lanes per
    thread)].  The roofline time is the slower of the HBM time (2 B / 8 bytes
    per attempt at the measured copy bandwidth) and the integer time (each
    part at its int_bound); frac = roofline time / measured time."""
    hbm = peaks["hbm_gbs"]
    alg_bytes = sum(a * 2.0 * rsos_bits(N) / 8.0 for a, N, _ in parts)
    attempts = sum(a for a, _, _ in parts)
    t_hbm = alg_bytes / (hbm * 1e9)
    bounds = [int_bound(N, w, int_peaks) for _, N, w in parts]
    t_int = sum(a / b["attempts_per_s"] for (a, _, _), b in zip(parts, bounds))
    if t_hbm >= t_int:
        achieved = alg_bytes / seconds / 1e9
        line = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm}
    else:
        achieved = attempts / seconds
        peak = attempts / t_int
        line = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "attempts/s", "frac": achieved / peak,
                "peak_note": "integer-pipe bound from measured lop3 and Philox rates (int_bound)"}
    line.update({"peak_source": peak_src, "algorithmic_bytes": alg_bytes,
                 "hbm_bound_attempts_per_s": attempts / t_hbm, "int_bound_attempts_per_s": attempts / t_int,
                 "int_bound": bounds[0] if len(bounds) == 1 else {"pipes": sorted({b["pipe"] for b in bounds})}})
    line.update(extra)
    return line


def kernel_hash(kind: str) -> str:
    h = hashlib.sha256()
    for rel in KERNELS[kind]["sources"]:
        with open(os.path.join(ROOT, CSRC + rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, kind: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary of the workload, if it was taken on the current kernel source."""
    try:
        text = open(os.path.join(ROOT, "profiles", PROFILES[workload])).read()
    except (OSError, KeyError):
        return None
    m = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_hash(kind):
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
    R.rsos_sweep(h, 50 if L <= 8192 else 3, stream=stream)
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_kernel_sweeps = 200 if L <= 8192 else 50
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
    kind = "general" if W["tiling"] == 1 else "persistent"
    # launches in the kernel-timing region: one persistent launch, or four
    # phase launches per sweep
    lps = KERNELS[kind]["launches_per_sweep"]
    n_launch = lps * n_kernel_sweeps if lps else 1
    per_launch_ms = launch_ms / n_launch
    launches_per_job = launches[0]
    if rank != 0:
        return
    int_peaks = measure_int_peaks(R, stream)
    lanes = lanes_per_thread(W["N"], S)
    wt = "uint64_t" if lanes == 64 else "uint32_t"
    kname = (f"rsos::general_phase_kernel<{W['N']}, {wt}>" if kind == "general"
             else f"rsos::persistent_kernel<{W['N']}, {wt}, 4>")
    attempts_per_launch = float(L) * L * S * n_kernel_sweeps / n_launch
    roof = roofline_of([(attempts_per_launch, W["N"], lanes)], per_launch_ms / 1e3, peaks, peak_src, int_peaks,
                       traffic=profiled_traffic(args.workload_key, kind), kernel=kname, launch_ms=per_launch_ms,
                       sweeps_per_launch=n_kernel_sweeps / n_launch,
                       algorithmic_bytes_per_launch=attempts_per_launch * 2 * rsos_bits(W["N"]) / 8)
    cpu = cpu_baseline(L, W["N"], W["tile"], seed, tiling=W["tiling"]) if world == 1 else None
    lanes_note = f"inputs larger than L2 ({L * L * S * rsos_bits(W['N']) / 8 / 2 ** 20:.0f} MiB lattice per job)"
    line = {
        "metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": f"{'u64' if lanes == 64 else 'u32'} (bit-sliced int)",
        "data": "synthetic",
        "config": dict(W, parallelism=f"replicas{world}", l2=lanes_note, seed=seed),
        "e2e": {"value": e2e_value, "unit": "attempts/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": (len(times)) * S * 4 * 8 + 8},
        "roofline": roof,
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


def cpu_baseline(L, N, T, seed, target_s: float = 12.0, tiling: int = 0, mem_bytes: float = 16e9):
    """The oracle, as it stands, on the host cores: DT sweeps of the
    workload's lattice for up to one lane per core (fewer where the int64
    height fields would exceed mem_bytes), repeated until about ``target_s``
    seconds of CPU work or 8 sweeps."""
    import oracle as O
    cores = os.cpu_count() or 1
    Tx, Ty = _edges(T)
    p = O.Params(L=L, N=N, Tx=Tx, Ty=Ty, seed=seed, tiling=tiling)
    n = int(max(1, min(cores, mem_bytes // (8.0 * L * L))))
    lanes = list(range(n))
    h = O.flat(L, n)
    done, t0 = 0, time.perf_counter()
    while True:
        O.sweeps(p, h, lanes, done, 1, threads=cores)
        done += 1
        el = time.perf_counter() - t0
        if el > target_s or done >= 8:
            break
    value = float(L) * L * n * done / el
    return {"value": value, "unit": "attempts/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} DT sweep(s) of L={L}, N={N}, {n} lanes, {cores} threads, from the flat start"}


def cpu_baseline_jobs(jobs, target_s: float = 12.0):
    """The oracle on a bounded sample of a job list: one DT sweep of each job
    in order (lanes 0..min(cores, S)-1), until about ``target_s`` seconds."""
    import oracle as O
    cores = os.cpu_count() or 1
    attempts, done, t0 = 0.0, 0, time.perf_counter()
    for j in jobs:
        n = min(cores, j["surfaces"])
        O.sweeps(O.Params(L=j["L"], N=j["N"], Tx=8, Ty=8, seed=j["seed"]), O.flat(j["L"], n), list(range(n)), 0, 1,
                 threads=cores)
        attempts += float(j["L"]) * j["L"] * n
        done += 1
        if time.perf_counter() - t0 > target_s:
            break
    el = time.perf_counter() - t0
    return {"value": attempts / el, "unit": "attempts/s", "cores": cores, "kind": "oracle",
            "sample": f"one DT sweep of each of the first {done} jobs (up to {cores} lanes each) from the flat start"}


def run_batched(args):
    """Batched workload: 256 independent jobs (L uniform in {256..4096}, N in
    {1, 2}, 64 surfaces, t_max log-uniform in [1e3, 1e4] sweeps, seeds =
    job index), one multi-job persistent launch per class, captured in a CUDA
    graph; each job's width is measured exactly at its t_max.  One step = the
    whole batch through the public API: rsos_batch_create (the library
    allocates), rsos_batch_run, polling, the read-back of every job's W^2 and
    rsos_batch_free.  value = attempts / device time of rsos_batch_run (CUDA
    events); e2e = attempts / wall time of the whole step."""
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
    d2h = [0]

    def one_batch(tm=None):
        w0 = time.perf_counter()
        b = R.rsos_batch_create(params, tm or tmax)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        R.rsos_batch_run(b, stream)
        ev1.record(stream)
        done = set()
        while len(done) < len(jobs):
            _, ids = R.rsos_batch_poll(b)
            done |= set(ids)
        w2 = []
        for k in range(len(jobs)):
            w2.append(R.rsos_read_series(R.rsos_batch_job(b, k), jobs[k]["surfaces"], 2)[3][-1])
        R.rsos_batch_free(b)
        wall = time.perf_counter() - w0
        d2h[0] = sum(x.nbytes * 3 + 8 for x in w2)  # t, sum h, sum h^2, W^2 per surface
        return ev0.elapsed_time(ev1), wall, [float(x.mean()) for x in w2[::64]]

    # warm-up: the same batch with t_max / 100 (compiles plans, warms clocks)
    warm_tmax = [max(1, t // 100) for t in tmax]
    for _ in range(args.warmup):
        one_batch(warm_tmax)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    total_ms, total_wall = 0.0, 0.0
    for _ in range(args.steps):
        ms, wall, w2 = one_batch()
        total_ms += ms
        total_wall += wall
    clk = clocks.stop()
    value = attempts * args.steps / (total_ms / 1e3)
    e2e_value = attempts * args.steps / total_wall

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
    classes = {}
    for j, t in zip(jobs, tmax):
        c = classes.setdefault(f"L{j['L']}_N{j['N']}", {"jobs": 0, "attempts": 0.0, "alone_s": 0.0})
        c["jobs"] += 1
        c["attempts"] += float(j["L"]) * j["L"] * j["surfaces"] * t
        c["alone_s"] += j["L"] * j["L"] * j["surfaces"] * t / rates[(j["L"], j["N"])]
    for (L, N), r in rates.items():
        classes[f"L{L}_N{N}"]["alone_rate"] = r
    peaks, peak_src = measured_peaks()
    int_peaks = measure_int_peaks(R, stream)
    parts = [(float(j["L"]) * j["L"] * j["surfaces"] * t, j["N"], 64 if geometry[(j["L"], j["N"])][0] == 2 else 32)
             for j, t in zip(jobs, tmax)]
    roof = roofline_of(parts, total_ms / args.steps / 1e3, peaks, peak_src, int_peaks,
                       traffic=None, kernel="rsos::persistent_multi_kernel (all classes of the batch)",
                       note="whole batch: algorithmic bytes of every job over the device time of rsos_batch_run")
    cpu = cpu_baseline_jobs(jobs)
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64/u32 (bit-sliced int)", "data": "synthetic",
        "e2e": {"value": e2e_value, "unit": "attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h[0],
                "how": "wall time of create + run + poll + read-back of every job + free"},
        "roofline": roof, "cpu_baseline": cpu, "int_peaks": int_peaks,
        "plain_equivalent": {"value": plain_equiv, "unit": "attempts/s", "ratio": value / plain_equiv,
                             "how": "the same jobs run one at a time, each at its own (L, N) single-job rate "
                                    "with the same autotuned geometry",
                             "classes": classes},
        "config": {"workload": f"batched: 256 jobs, L in {{256..4096}}, N in {{1,2}}, 64 surfaces, t_max in "
                               f"[1e3,1e4]{'' if scale == 1 else f'/{scale}'} sweeps, PCG64 seed 2016; one multi-job "
                               "persistent launch per class in a CUDA graph; execution geometry per (L, N) from "
                               "rsos_autotune",
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
    second) bound the run; the JSON line states them.  The server is the
    public API a user calls, so value and e2e are the same wall-clock rate."""
    import torch

    import paper_1605_02620_gb300 as R
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
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    server = Server(hbm_budget=args.serve_budget, epoch_s=args.serve_epoch, stream=stream, tune=True)
    rep = server.run(reqs)
    clk = clocks.stop()
    s = rep.summary()
    by_id = {r.rid: r for r in reqs}
    done = [by_id[r.rid] for r in rep.results if r.status == "done"]
    peaks, peak_src = measured_peaks()
    int_peaks = measure_int_peaks(R, stream)
    geo = {}
    for q in done:
        if (q.L, q.N) not in geo:
            geo[(q.L, q.N)] = server._params(q).words_per_thread
    parts = [(float(q.L) * q.L * q.surfaces * q.t_max, q.N, 64 if geo[(q.L, q.N)] == 2 else 32) for q in done]
    busy = rep.gpu_busy_s if rep.gpu_busy_s > 0 else rep.wall_s
    roof = roofline_of(parts, busy, peaks, peak_src, int_peaks, traffic=None,
                       kernel="rsos::persistent_multi_kernel (rsos_advance epochs)",
                       note="algorithmic bytes of every served job over the busy time of the epochs "
                            "(rsos_advance calls); frac_wall over the whole run",
                       frac_wall=None)
    roof["frac_wall"] = roof["frac"] * busy / rep.wall_s
    load = s["offered_attempts_per_s"] / s["attempts_per_busy_s"] if s["attempts_per_busy_s"] else None
    label = args.serve_label or ("overloaded" if load and load > 1.0 else "under capacity")
    cpu = cpu_baseline_jobs(jobs)
    d2h = sum(q.surfaces * 3 * 8 + 8 for q in done)
    print(json.dumps({
        "metric": METRIC, "value": s["attempts_per_s"], "unit": "attempts/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": rep.wall_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64/u32 (bit-sliced int)", "data": "synthetic",
        "e2e": {"value": s["attempts_per_s"], "unit": "attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h,
                "how": "the server loop itself: admission (rsos_init), epochs, read-back and release, wall clock"},
        "roofline": roof, "cpu_baseline": cpu, "int_peaks": int_peaks,
        "config": {"workload": f"served ({label}): {len(reqs)} Poisson requests at {args.serve_rate}/s, L=2^(8..13), "
                               f"N in 1..4, 64 surfaces, t_max in [1e2,1e4]"
                               f"{'' if args.serve_scale == 1 else f'/{args.serve_scale}'} sweeps, PCG64 seed 2017",
                   "hbm_budget": args.serve_budget, "epoch_s": args.serve_epoch,
                   "offered_load_over_capacity": load,
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
    ap.add_argument("--L", type=int, default=0,
                    help="lattice edge (reduced values only for profiling captures of large workloads)")
    ap.add_argument("--workload", default="ms-n1", choices=["ms-n1", "irregular", "step-height", "batched", "served"])
    ap.add_argument("--N", type=int, default=1, choices=[1, 2, 4], help="step bound of the step-height workload")
    ap.add_argument("--batch-scale", type=int, default=1,
                    help="divide the batched jobs' t_max by this factor (profiling / quick checks)")
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-scale", type=int, default=1)
    ap.add_argument("--serve-budget", type=int, default=200 << 30)
    ap.add_argument("--serve-epoch", type=float, default=0.02)
    ap.add_argument("--serve-label", default="", help="label of the served run (e.g. ~70%% load)")
    ap.add_argument("--quick", action="store_true",
                    help="profiling capture: timed steps only (no kernel timing, e2e or CPU baseline)")
    args = ap.parse_args()
    args.workload_key = args.workload
    if args.workload in ("irregular", "step-height"):
        WORKLOAD.clear()
        WORKLOAD.update(WORKLOAD_IRREGULAR if args.workload == "irregular" else step_height_workload(args.N))
        if args.workload == "step-height":
            args.workload_key = f"step-height-{args.N}"
        if "--sweeps" not in sys.argv:
            args.sweeps = WORKLOAD["sweeps"]
        if "--measurements" not in sys.argv:
            args.measurements = WORKLOAD["measurements"]
    if args.L and args.L != WORKLOAD["L"]:
        WORKLOAD["workload"] += f" [lattice reduced to L={args.L} for profiling]"
        WORKLOAD["L"] = args.L
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
