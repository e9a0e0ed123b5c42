"""Benchmark: batched env step + render (frames/s) on GB300.

Workload: 4096 envs, 32 x 32 random DFS key-door mazes, 64 x 64 RGB frames,
horizon 500 with auto-reset, 10,000 steps of uniform random actions (seed 1).
A step moves, collides, picks up, rewards, resets and renders all envs. The
timed path runs the pre-drawn action stream through jx_rollout, 128 steps per
launch; every step writes its frames into slot (step mod 128) of a 6.4 GB
rollout buffer, so the frame stream never fits the 126 MB L2 and every byte
goes to HBM. The single-step entry point (jx_step, CUDA graph of 128
launches) is timed on the same workload beside it, and its per-call latency
gives p50 / p99.

Prints one JSON line. ``--impl reference`` times the FP64 CPU oracle on the
same workload instead (the method's only other implementation here).
"""

from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s incl. render (frames/s) at 64x64 RGB"
GRAPH_STEPS = 128  # default launches per CUDA graph = rollout buffer slots
KERNEL_SOURCES = ["paper_2605_19926_gb300/csrc/jx_device.cuh", "paper_2605_19926_gb300/csrc/jx_kernels.cu",
                  "paper_2605_19926_gb300/csrc/jx_internal.h"]
BATCH_KERNEL_SOURCES = ["paper_2605_19926_gb300/csrc/jx_device.cuh", "paper_2605_19926_gb300/csrc/jx_batch_kernels.cu",
                        "paper_2605_19926_gb300/csrc/jx_internal.h"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
TRAFFIC_UNEVEN_FILE = os.path.join(ROOT, "profiles", "traffic_uneven.json")
TRAFFIC_LARGE_FILE = os.path.join(ROOT, "profiles", "traffic_large.json")


def kernel_code(text: str) -> str:
    """Source text without comments and blank space: edits to comments leave
    the compiled kernel, and so the traffic record, valid."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_sha(sources=None) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES if sources is None else sources:
        h.update(kernel_code(open(os.path.join(ROOT, f)).read()).encode())
    return h.hexdigest()[:16]


def tiling_key(t, sides) -> tuple:
    """What of a batched-kernel tiling decides the DRAM bytes on maps of the
    given sides: which maps are bit planes (ray hits then read the hit cell's
    type from HBM). Warps per block, rays per lane, rows per block and staging
    buffers change how the same frames are written, not which bytes move."""
    b = int(t[2])
    return tuple(b > 0 and s >= b and s % 8 == 0 for s in sides)


def recorded_traffic(n_envs: int, launch_steps: int, path: str = TRAFFIC_FILE, sources=None, tiling=None):
    """DRAM bytes of one launch from the ncu record, scaled from the captured
    launch by the env-steps processed; None when the record is missing, was
    taken on other kernel code or another batched-kernel tiling, or is for
    another env count without saying that its traffic grows in proportion to
    the env-steps."""
    if not os.path.exists(path):
        return None
    tf = json.load(open(path))
    if tf.get("kernel_source_sha") != kernel_source_sha(sources):
        return None
    if "tiling" in tf:
        sides = tf.get("map_sides", [])
        if tiling is None or tiling_key(tf["tiling"], sides) != tiling_key(tiling, sides):
            return None
    if tf.get("n_envs") != n_envs and not tf.get("scales_with_env_steps"):
        return None
    return tf["dram_bytes_per_env_step"] * n_envs * launch_steps


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def shard_config(cfg: dict, rank: int) -> dict:
    """Each rank steps its own independent envs (weak scaling): same shape, its own seed."""
    out = dict(cfg)
    out["seed"] = int(cfg["seed"]) + rank
    return out


STATE_READ = 2 + 2 + 4 + 4 + 4 + 4 + 2 + 4 + 4 + 1 + 12 + 1  # cells, fracs, cos/sin, turn, t, episode, flags,
# objects, sprite count (+ the sprite table, K * 9 bytes)
STATE_WRITE = 2 + 2 + 4 + 4 + 2 + 4 + 1  # cells, fracs, turn, t, flags
STEP_IO = 1 + 4 + 1  # action, reward, done


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The slowest rank's time: the job is done when every rank is."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, n_envs_per_rank: int, steps: int, t_max_ms: float) -> float:
    """Whole-job env-steps/s: every rank steps its own n_envs for `steps` steps."""
    return world * n_envs_per_rank * steps / (t_max_ms / 1e3)


def algorithmic_bytes_per_env_step(cfg: dict) -> int:
    """Compulsory HBM bytes of one jx_step per env: the frame written, the state
    read and written, action, reward and done. The map (re-read from L2 every
    step) and episode regeneration (once per horizon) are excluded."""
    H, W, K = cfg["frame_h"], cfg["frame_w"], cfg["max_sprites"]
    return 3 * H * W + STATE_READ + 9 * K + STATE_WRITE + STEP_IO


def rollout_bytes(cfg: dict, n_envs: int, steps: int) -> int:
    """Compulsory HBM bytes of one jx_rollout launch: per env and step the frame,
    action, reward and done; per env the state read once and written once."""
    H, W, K = cfg["frame_h"], cfg["frame_w"], cfg["max_sprites"]
    return n_envs * steps * (3 * H * W + STEP_IO) + n_envs * (STATE_READ + 9 * K + STATE_WRITE)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def time_oracle(cfg: dict, n_envs: int, n_steps: int, seed: int, nthreads: int) -> tuple[float, int]:
    """Oracle env-steps/s over n_envs x n_steps of the workload (frames rendered)."""
    import oracle

    ocfg = oracle.make_config(**cfg)
    from paper_2605_19926_gb300 import inputs

    envs = oracle.generate(ocfg, np.arange(n_envs), nthreads=nthreads)
    acts = [inputs.actions(seed, s, n_envs) for s in range(n_steps)]
    t0 = time.perf_counter()
    for s in range(n_steps):
        oracle.step(ocfg, np.arange(n_envs), envs, acts[s], frames=True, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return n_envs * n_steps / dt, nthreads


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, cfg: dict):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    # envs per step: the whole batch while the run stays near a minute of
    # oracle work (~3.6e7 env-steps at the measured ~6.7e5 env-steps/s on 16
    # cores), fewer for long runs, never under 256
    n_envs = args.ref_envs or max(256, min(cfg["n_envs"], int(3.6e7 // max(1, args.steps + args.warmup))))
    cores = cpu_cores()
    # W untimed warm-up steps, then K steps, each over a bounded sample of the envs
    time_oracle(cfg, n_envs, args.warmup, seed=cfg["seed"], nthreads=cores)
    value, used = time_oracle(cfg, n_envs, args.steps, seed=cfg["seed"], nthreads=cores)
    t_total = n_envs * args.steps / value  # the timed stepping, as in `value`
    steps_total = args.steps
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": args.gpus,
        "steps": steps_total, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / steps_total,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "4096 envs, 32x32 DFS key-door mazes, 64x64 RGB, horizon 500, random actions",
                   "sample_envs": n_envs},
        "cpu_baseline": {"value": value, "unit": "env-steps/s", "cores": used, "kind": "oracle",
                         "sample": f"{n_envs} envs x {steps_total} steps of the workload (frames rendered)"},
        "e2e": {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def tiling_dict(t) -> dict:
    """A launch choice as JSON: all zero means the env's own kernel."""
    names = ("warps_per_block", "cols_per_lane", "bits_min_side", "max_rows_per_block", "staging_buffers")
    d = dict(zip(names, t.as_tuple()))
    d["kernel"] = "env kernel" if not any(t.as_tuple()) else "batched kernel"
    return d


def uneven_bytes_per_env_step(groups: list) -> float:
    """Mean compulsory HBM bytes per env-step of an uneven batch (as for one env group)."""
    tot = sum(g["n_envs"] * algorithmic_bytes_per_env_step(g) for g in groups)
    return tot / sum(g["n_envs"] for g in groups)


def run_uneven(args):
    """Uneven batching: 16,384 envs of 16 (map side, frame size) groups in one
    persistent launch per rollout; fixed tiles against autotuned tiles, and the
    autotuned step sequence replayed as a CUDA graph."""
    import torch

    from paper_2605_19926_gb300 import build, inputs

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2605_19926_gb300 import jx

    groups = inputs.uneven_groups(n_envs=args.uneven_envs, seed=2 + rank)
    envs = [jx.Env(c, local) for c in groups]
    pinned = parse_tiling(jx, args.tiling)
    batch = jx.Batch(envs, pinned)
    N, F = batch.n, batch.frame_bytes
    dev = torch.device("cuda", local)
    T = args.uneven_slots
    K = max(T, (args.steps // T) * T)
    acts = torch.from_numpy(inputs.action_stream(7 + rank, K + T, N)).to(dev)
    frames = torch.empty((T, F), dtype=torch.uint8, device=dev)  # T x 0.38 GB > L2
    rewards = torch.empty((T, N), dtype=torch.float32, device=dev)
    dones = torch.empty((T, N), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def timed_rollouts() -> tuple[float, int]:
        with torch.cuda.stream(stream):
            batch.reset(frames[0], stream)
            batch.rollout(acts[:T], frames, rewards, dones, stream)  # warm-up
        stream.synchronize()
        n0 = batch.launch_count()
        if world > 1:
            torch.distributed.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for c in range(K // T):
                batch.rollout(acts[T + c * T: T + (c + 1) * T], frames, rewards, dones, stream)
            e1.record(stream)
        stream.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), world, dev), batch.launch_count() - n0

    fixed_ms, _ = timed_rollouts()
    fixed_tiling = batch.tiling
    t_tune = time.perf_counter()
    trials = [] if pinned is not None else batch.autotune(mode=1, steps=T, max_trials=args.tune_trials,
                                                          stream=stream)
    tune_s = time.perf_counter() - t_tune
    tuned = batch.tiling
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    tuned_ms, launches = timed_rollouts()
    clk = clocks.stop()
    # the same steps as a CUDA graph of T single-step launches, replayed
    graph = batch.capture(acts[T: 2 * T], frames, rewards, dones)
    with torch.cuda.stream(stream):
        batch.reset(frames[0], stream)
        graph.launch(stream)
    stream.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        g0.record(stream)
        for c in range(K // T):
            graph.launch(stream)
        g1.record(stream)
    stream.synchronize()
    graph_ms = max_over_ranks(g0.elapsed_time(g1), world, dev)
    graph.close()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    bpes = uneven_bytes_per_env_step(groups)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, peak_src = 6800.0, "fallback"
    if os.path.exists(peaks_path):
        peak, peak_src = float(json.load(open(peaks_path))["hbm_gbs"]), "measured"

    def leg(ms, tiling):
        v = world * N * K / (ms / 1e3)
        gbs = N * K * bpes / (ms / 1e3) / 1e9 / world
        return {"value": v, "ms_per_step": ms / K, "achieved_gbs": gbs, "frac": gbs / peak,
                "tiling": tiling_dict(tiling)}

    shape = batch.launch_shape()
    tuned_leg = leg(tuned_ms, tuned)
    line = {
        "metric": "env-steps/s incl. render (frames/s), uneven batch", "value": tuned_leg["value"],
        "unit": "env-steps/s", "n_gpus": world, "steps": K, "warmup": T, "ms_per_step": tuned_ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"{N:,} envs per GPU, random-wall rooms p=0.3, map side uniform in {{16,32,64,128}}, "
                               "square RGB frames uniform in {32,64,96,128}, 0-8 sprites, uniform random actions",
                   "groups": len(groups), "n_envs_per_gpu": N, "frame_bytes_per_step": F,
                   "parallelism": f"replicas x{world}",
                   "l2": f"frames written to a {T}-slot rollout buffer ({T * F / 1e9:.1f} GB) > L2",
                   "launch": {"grid": shape.grid, "block": shape.block, "smem_bytes": shape.smem,
                              "entry": "jx_batch_rollout", "steps_per_launch": T}},
        "roofline": {"bound": "hbm", "achieved": tuned_leg["achieved_gbs"], "peak": peak, "unit": "GB/s",
                     "frac": tuned_leg["frac"],
                     "traffic": recorded_traffic(N, T, TRAFFIC_UNEVEN_FILE, BATCH_KERNEL_SOURCES,
                                                 tuned.as_tuple()),
                     "peak_source": peak_src,
                     "algorithmic_bytes_per_env_step": bpes},
        "fixed_tiles": leg(fixed_ms, fixed_tiling), "autotuned": tuned_leg,
        "autotune": {"trials": len(trials), "seconds": tune_s, "mode": "rollout", "steps_per_trial": T},
        "graph_steps": {"value": world * N * K / (graph_ms / 1e3), "ms_per_step": graph_ms / K,
                        "how": f"jx_batch_capture of {T} jx_batch_step launches, replayed"},
        "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def parse_tiling(jx, text: str):
    """`w,c,b,r[,s]` -> a jx.Tiling (staging buffers default to 1), or None for ''."""
    if not text:
        return None
    t = jx.Tiling()
    vals = [int(v) for v in text.split(",")] + [1]
    (t.warps_per_block, t.cols_per_lane, t.bits_min_side, t.max_rows_per_block, t.staging_buffers) = vals[:5]
    return t


def run_large(args):
    """Large scale: 65,536 envs of 128 x 128 mazes with 8 x 8 rooms, 16 sprite
    slots, 128 x 128 RGB frames plus the 4-frame grayscale stack written in the
    same pass, horizon 500, `--steps` (1000) steps of uniform random actions in
    rollout launches of `--large-slots` steps."""
    import torch

    from paper_2605_19926_gb300 import build, inputs

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2605_19926_gb300 import jx

    cfg = shard_config(inputs.large_scale(args.large_envs), rank)
    N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    dev = torch.device("cuda", local)
    env = jx.Env(cfg, local)
    tuned = None
    if args.tiling:
        env.tiling = parse_tiling(jx, args.tiling)  # the batched kernel with this tiling
    elif not args.no_autotune:
        # the env's own kernel against the batched kernel's tilings, before timing
        tuned = env.autotune(mode=1, steps=args.large_slots, max_trials=args.tune_trials)
    T = args.large_slots
    K = max(T, (args.steps // T) * T)
    acts = torch.from_numpy(inputs.action_stream(cfg["seed"], K + T, N)).to(dev)
    frames = torch.empty((T, N, H, W, 3), dtype=torch.uint8, device=dev)
    rewards = torch.empty((T, N), dtype=torch.float32, device=dev)
    dones = torch.empty((T, N), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    t_reset = time.perf_counter()
    with torch.cuda.stream(stream):
        env.reset(frames[0], stream)
    stream.synchronize()
    reset_s = time.perf_counter() - t_reset
    with torch.cuda.stream(stream):
        env.rollout(acts[:T], frames, rewards, dones, stream)  # warm-up
    stream.synchronize()
    n0 = env.launch_count()
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for c in range(K // T):
            env.rollout(acts[T + c * T: T + (c + 1) * T], frames, rewards, dones, stream)
        e1.record(stream)
    stream.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    launches = env.launch_count() - n0
    n_done = int(dones.sum().item())
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    gray = H * W  # one plane per env-step (all four at an episode start)
    bpes = algorithmic_bytes_per_env_step(cfg) + gray
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, peak_src = 6800.0, "fallback"
    if os.path.exists(peaks_path):
        peak, peak_src = float(json.load(open(peaks_path))["hbm_gbs"]), "measured"
    gbs = N * K * bpes / (ms / 1e3) / 1e9
    shape = env.launch_shape()
    line = {
        "metric": "env-steps/s incl. render (frames/s), 128x128 RGB + gray stack", "value": world * N * K / (ms / 1e3),
        "unit": "env-steps/s", "n_gpus": world, "steps": K, "warmup": T, "ms_per_step": ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"{N} envs per GPU, 128x128 DFS mazes with 8x8 open rooms, 16 sprite slots (key, goal, "
                               "0-14 distractors), 128x128 RGB + 4-frame grayscale stack in the same pass, horizon 500, "
                               "uniform random actions",
                   "parallelism": f"replicas x{world}",
                   "l2": f"frames written to a {T}-slot rollout buffer ({T * N * H * W * 3 / 1e9:.1f} GB) > L2",
                   "launch": {"grid": shape.grid, "block": shape.block, "smem_bytes": shape.smem,
                              "entry": "jx_rollout", "steps_per_launch": T}},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                     "traffic": recorded_traffic(N, T, TRAFFIC_LARGE_FILE, BATCH_KERNEL_SOURCES,
                                                 env.tiling.as_tuple()),
                     "peak_source": peak_src, "algorithmic_bytes_per_env_step": bpes},
        "reset_seconds": reset_s, "episode_ends_in_last_launch": n_done,
        "tiling": tiling_dict(env.tiling),
        "autotune_trials": len(tuned) if tuned else 0,
        "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_serve(args):
    """Serving: 64 actor groups submit step requests with Poisson arrivals
    (mean gap 2 ms) to the continuous-batching server. Each group runs
    sessions of `--session-steps` requests; a session's batch is log-uniform
    in [16, 4096] envs of 32x32 or 64x64 key-door mazes, 64x64 RGB. Sessions
    are admitted under a 40 GB state+frame budget. Reports p50 / p99 request
    latency (submit to completion) and aggregate env-steps/s."""
    import concurrent.futures as cf
    import heapq

    import torch

    from paper_2605_19926_gb300 import build, inputs

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2605_19926_gb300 import jx

    seed = 3 + rank
    n_actors, duration, warm = args.actors, args.serve_seconds, min(2.0, args.serve_seconds / 4)
    server = jx.Server(budget_bytes=int(args.budget_gb * 1e9), max_sessions=4 * n_actors, max_inflight=4,
                       max_map_side=64, device=local)
    pool = cf.ThreadPoolExecutor(max_workers=4)
    session = [None] * n_actors  # open Session or None
    opening = [None] * n_actors  # future of a pending open
    left = [0] * n_actors
    k_next = [0] * n_actors
    acts = [None] * n_actors
    gaps = [inputs.arrival_gaps(seed, a, 1 << 16) for a in range(n_actors)]
    gi = [0] * n_actors
    heap = [(float(gaps[a][0]), a) for a in range(n_actors)]
    heapq.heapify(heap)
    for a in range(n_actors):
        gi[a] = 1
    t0 = time.perf_counter()
    lat_mark = None
    stats_mark = None
    submitted = 0
    while heap:
        t_rel, a = heapq.heappop(heap)
        if t_rel > duration:
            break
        while time.perf_counter() - t0 < t_rel:
            pass
        if lat_mark is None and t_rel >= warm:
            server.latencies()  # drop the warm-up requests
            stats_mark = (time.perf_counter(), server.stats())
            lat_mark = True
        if session[a] is None and opening[a] is not None and opening[a].done():
            session[a] = opening[a].result()
            opening[a] = None
            if session[a] is not None:
                left[a] = args.session_steps
                n = session[a].n
                acts[a] = np.random.default_rng([seed, a, k_next[a]]).integers(0, 7, size=(8, n), dtype=np.uint8)
        if session[a] is not None:
            session[a].submit(acts[a][left[a] % 8])
            submitted += 1
            left[a] -= 1
            if left[a] == 0:
                session[a].close()
                session[a] = None
        elif opening[a] is None:
            cfg = inputs.serving_session(seed, a, k_next[a])
            k_next[a] += 1
            opening[a] = pool.submit(server.try_open, cfg)
        heapq.heappush(heap, (t_rel + float(gaps[a][gi[a] % len(gaps[a])]), a))
        gi[a] += 1
    t_end = time.perf_counter()
    st_end = server.stats()
    lat = server.latencies()
    pool.shutdown(wait=True)
    t_stats0, st0 = stats_mark
    window = t_end - t_stats0
    env_steps = st_end["env_steps"] - st0["env_steps"]
    reqs = st_end["requests_done"] - st0["requests_done"]
    launches = st_end["launches"] - st0["launches"]
    groups = st_end["groups_launched"] - st0["groups_launched"]
    server.close()
    value = env_steps / window
    p50 = float(np.percentile(lat, 50)) * 1e3 if len(lat) else None
    p99 = float(np.percentile(lat, 99)) * 1e3 if len(lat) else None
    tot = max_over_ranks(window * 1e3, world, torch.device("cuda", local))
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    line = {
        "metric": "env-steps/s incl. render (frames/s), served requests", "value": value * world,
        "unit": "env-steps/s", "n_gpus": world, "steps": int(reqs), "warmup": 0,
        "ms_per_step": tot / max(1, reqs), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"{n_actors} actor groups, Poisson arrivals (mean gap 2 ms), sessions of "
                               f"{args.session_steps} requests, batch log-uniform in [16, 4096] envs, 32x32 or 64x64 "
                               "key-door mazes, 64x64 RGB, continuous batching",
                   "budget_gb": args.budget_gb, "seconds": duration, "measured_seconds": window,
                   "max_inflight_launches": 4},
        "p50_step_ms": p50, "p99_step_ms": p99,
        "requests_per_s": reqs / window, "submitted_per_s": submitted / (t_end - t0),
        "mean_sessions_per_launch": groups / max(1, launches), "launches": int(launches),
        "server": {k: st_end[k] for k in ("peak_bytes_in_use", "budget_bytes", "peak_sessions",
                                          "peak_inflight_launches", "rejected_opens")},
        "roofline": None, "cpu_baseline": None,
        "e2e": {"value": value * world, "unit": "env-steps/s", "h2d_bytes_per_step": None, "d2h_bytes_per_step": 0,
                "how": "host actions submitted per request through jx_server_submit; results stay on the device"},
        "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=16)
    ap.add_argument("--impl", default="jx", choices=["jx", "reference"])
    ap.add_argument("--n-envs", type=int, default=4096)
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--latency-steps", type=int, default=300)
    ap.add_argument("--cpu-envs", type=int, default=4096)
    ap.add_argument("--cpu-steps", type=int, default=600)
    ap.add_argument("--ref-envs", type=int, default=0, help="reference arm: envs per step (0: sized to the run)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=1000)
    ap.add_argument("--ring-slots", type=int, default=GRAPH_STEPS,
                    help="rollout buffer slots = launches per CUDA graph (smaller for profiling captures)")
    ap.add_argument("--workload", default="mazes", choices=["mazes", "uneven", "serve", "large"],
                    help="mazes: 4096 key-door mazes (the headline); uneven: 16,384 envs of mixed sizes; "
                         "serve: the continuous-batching step server under Poisson request arrivals")
    ap.add_argument("--actors", type=int, default=64)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--session-steps", type=int, default=250)
    ap.add_argument("--budget-gb", type=float, default=40.0)
    ap.add_argument("--large-envs", type=int, default=65536)
    ap.add_argument("--large-slots", type=int, default=8, help="steps per rollout launch of the large workload")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip jx_autotune before timing (the env's own kernel with its fixed tiles)")
    ap.add_argument("--uneven-slots", type=int, default=16, help="steps per rollout launch of the uneven batch")
    ap.add_argument("--uneven-envs", type=int, default=16384)
    ap.add_argument("--tiling", default="",
                    help="uneven batch and large scale: w,c,b,r[,s] batched-kernel tiling to use instead of autotuning")
    ap.add_argument("--tune-trials", type=int, default=1000)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.workload == "large" and args.impl == "jx":
        if args.steps == ap.get_default("steps"):
            args.steps = 1000
        run_large(args)
        return
    if args.workload == "serve" and args.impl == "jx":
        run_serve(args)
        return
    if args.workload == "uneven" and args.impl == "jx":
        if args.steps == ap.get_default("steps"):
            args.steps = 512
        run_uneven(args)
        return

    from paper_2605_19926_gb300 import inputs

    base_cfg = inputs.batched_keydoor_mazes(args.n_envs)
    if args.impl == "reference":
        run_reference(args, base_cfg)
        return

    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2605_19926_gb300 import build

    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2605_19926_gb300 import jx

    cfg = shard_config(base_cfg, rank)
    N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    dev = torch.device("cuda", local)
    env = jx.Env(cfg, local)
    ring = args.ring_slots
    tuned = None
    if not args.no_autotune:
        # the env's own kernel against the batched kernel's tilings, before timing
        tuned = env.autotune(mode=1, steps=ring, max_trials=args.tune_trials)
    total_steps = args.warmup + args.steps
    # inputs resident in HBM before timing: the whole action stream
    acts_host = inputs.action_stream(cfg["seed"], total_steps, N)
    acts = torch.from_numpy(acts_host).to(dev)
    ring_acts = torch.empty((ring, N), dtype=torch.uint8, device=dev)
    frames = torch.empty((ring, N, H, W, 3), dtype=torch.uint8, device=dev)  # 6.4 GB rollout buffer at 128 slots
    rewards = torch.empty((ring, N), dtype=torch.float32, device=dev)
    dones = torch.empty((ring, N), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        env.reset(frames[0], stream)
        for s in range(args.warmup):
            env.step(acts[s], frames[s % ring], rewards[s % ring], dones[s % ring], stream)
    stream.synchronize()

    # single-step entry point: a CUDA graph of `ring` jx_step launches
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        for i in range(ring):
            env.step(ring_acts[i], frames[i], rewards[i], dones[i], torch.cuda.current_stream())
    torch.cuda.synchronize()
    # the capture itself ran nothing; the env state is still after the warm-up

    # timed region: the whole action stream in rollout launches of `ring` steps
    # (each launch writes one frame per env and step into the rollout buffer)
    n_full, rem = divmod(args.steps, ring)
    launches_before = env.launch_count()
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        s = args.warmup
        for c in range(n_full):
            env.rollout(acts[s: s + ring], frames, rewards, dones, stream)
            s += ring
        if rem:
            env.rollout(acts[s: s + rem], frames[:rem], rewards[:rem], dones[:rem], stream)
            s += rem
        ev1.record(stream)
    stream.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    gpu_launches = env.launch_count() - launches_before
    t_max = max_over_ranks(ms, world, dev)
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = t_max / args.steps
    value = job_value(world, N, args.steps, t_max)

    # the single-step entry point on the same workload (graph replays of `ring` launches)
    n_graph = max(1, min(n_full, 16))
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        g0.record(stream)
        for c in range(n_graph):
            ring_acts.copy_(acts[(args.warmup + c * ring) % (total_steps - ring + 1):][:ring], non_blocking=True)
            graph.replay()
        g1.record(stream)
    stream.synchronize()
    step_ms = g0.elapsed_time(g1) / (n_graph * ring)

    # per-step latency (eager launch + kernel, one step at a time)
    lat = []
    with torch.cuda.stream(stream):
        for i in range(args.latency_steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            env.step(acts[(args.warmup + i) % total_steps], frames[i % ring], rewards[i % ring], dones[i % ring],
                     stream)
            b.record(stream)
            b.synchronize()
            lat.append(a.elapsed_time(b))
    lat.sort()
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(0.99 * len(lat)))]

    # the plain method: one environment, one jx_step launch per step (16 x 16 rooms, 1000 steps)
    plain = None
    if rank == 0 and args.plain_steps > 0:
        pc = inputs.single_env_rooms()
        penv = jx.Env(pc, local)
        pa = torch.from_numpy(inputs.action_stream(pc["seed"], args.plain_steps, 1)).to(dev)
        pf = torch.empty((1, pc["frame_h"], pc["frame_w"], 3), dtype=torch.uint8, device=dev)
        pr = torch.empty(1, dtype=torch.float32, device=dev)
        pd = torch.empty(1, dtype=torch.uint8, device=dev)
        with torch.cuda.stream(stream):
            penv.reset(pf, stream)
            for i in range(8):
                penv.step(pa[i], pf, pr, pd, stream)
            p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p0.record(stream)
            for i in range(args.plain_steps):
                penv.step(pa[i], pf, pr, pd, stream)
            p1.record(stream)
        stream.synchronize()
        pms = p0.elapsed_time(p1)
        # its per-call latency, one step at a time with a host sync (as the batch's p50 / p99)
        plat = []
        with torch.cuda.stream(stream):
            for i in range(min(args.plain_steps, args.latency_steps)):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                penv.step(pa[i], pf, pr, pd, stream)
                b.record(stream)
                b.synchronize()
                plat.append(a.elapsed_time(b))
        plat.sort()
        plain = {"value": args.plain_steps / (pms / 1e3), "unit": "env-steps/s", "ms_per_step": pms / args.plain_steps,
                 "p50_step_ms": plat[len(plat) // 2] if plat else None,
                 "p99_step_ms": plat[min(len(plat) - 1, int(0.99 * len(plat)))] if plat else None,
                 "workload": f"1 env, 16x16 random rooms (p = 0.25), 64x64 RGB, {args.plain_steps} uniform random steps, "
                             "one jx_step launch per step"}
        penv.close()

    # end to end through the public host-buffer entry point
    h_act = torch.empty(N, dtype=torch.uint8).pin_memory()
    h_frames = torch.empty((N, H, W, 3), dtype=torch.uint8).pin_memory()
    h_rew = torch.empty(N, dtype=torch.float32).pin_memory()
    h_done = torch.empty(N, dtype=torch.uint8).pin_memory()
    for i in range(3):
        h_act.numpy()[:] = acts_host[i]
        env.step_host(h_act, h_frames, h_rew, h_done, stream)
    t0 = time.perf_counter()
    for i in range(args.e2e_steps):
        h_act.numpy()[:] = acts_host[(i + 3) % total_steps]
        env.step_host(h_act, h_frames, h_rew, h_done, stream)
    e2e_s = time.perf_counter() - t0
    e2e_value = world * N * args.e2e_steps / e2e_s  # every rank runs the same count; host clock per rank

    launch_steps = ring if n_full else rem
    bytes_per_launch = rollout_bytes(cfg, N, launch_steps)
    launch_ms = t_max / max(1, gpu_launches)
    achieved = bytes_per_launch / (launch_ms / 1e3) / 1e9
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, peak_src = 6800.0, "fallback"
    if os.path.exists(peaks_path):
        peak, peak_src = float(json.load(open(peaks_path))["hbm_gbs"]), "measured"
    traffic = recorded_traffic(N, launch_steps)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        import oracle

        oracle.build()
        v, cores = time_oracle(base_cfg, args.cpu_envs, args.cpu_steps, seed=base_cfg["seed"], nthreads=cpu_cores())
        # one core as well: the paper frames its CPU comparison per core
        n1, s1 = max(1, args.cpu_envs // 8), max(1, args.cpu_steps // 6)
        v1, _ = time_oracle(base_cfg, n1, s1, seed=base_cfg["seed"], nthreads=1)
        cpu = {"value": v, "unit": "env-steps/s", "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_envs} envs x {args.cpu_steps} steps of the workload (frames rendered)",
               "single_core": {"value": v1, "unit": "env-steps/s", "cores": 1,
                               "sample": f"{n1} envs x {s1} steps of the workload (frames rendered)"}}
    shape = env.launch_shape()
    line = {
        "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "4096 envs per GPU, 32x32 random DFS key-door mazes, 64x64 RGB uint8, horizon 500, "
                               "auto-reset, uniform random actions, seed 1",
                   "n_envs_per_gpu": N, "map_side": cfg["map_side"], "frame": f"{H}x{W}x3",
                   "parallelism": f"replicas x{world}",
                   "l2": f"frames written to a {ring}-slot rollout buffer ({ring * N * H * W * 3 / 1e9:.1f} GB) > L2",
                   "launch": {"grid": shape.grid, "block": shape.block, "smem_bytes": shape.smem,
                              "entry": "jx_rollout", "steps_per_launch": ring,
                              "tiling": tiling_dict(env.tiling), "autotune_trials": len(tuned) if tuned else 0}},
        "p50_step_ms": p50, "p99_step_ms": p99,
        "per_step_launch": {"value": world * N / (step_ms / 1e3), "unit": "env-steps/s", "ms_per_step": step_ms,
                            "how": f"jx_step, CUDA graph of {ring} launches"},
        "plain_one_env_per_launch": plain,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": bytes_per_launch},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "env-steps/s", "h2d_bytes_per_step": N,
                "d2h_bytes_per_step": N * H * W * 3 + 4 * N + N},
        "gpu_launches": gpu_launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
