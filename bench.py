"""Benchmark: batched env step + render (frames/s) on GB300.

Headline workload: 4096 envs, 32 x 32 random DFS key-door mazes, 64 x 64 RGB
frames, horizon 500 with auto-reset, uniform random actions (seed 1; the
paper times its environments under a uniform random policy, App. A.1). A step
moves, collides, picks up, rewards, resets and renders all envs.

The timed region runs `--steps` steps of the pre-drawn action stream through
jx_rollout, at most `--ring-slots` steps per launch; step s writes its frames
into slot (s mod ring) of a rollout buffer of at least four slots (>= 200 MB,
more than the 126 MB L2), so consecutive steps never reuse L2 lines. Beside
it, on the same workload:
  - per_step_launch: jx_step, one launch per step, as one CUDA graph of at
    least 128 launches, each reading its own row of the action stream (the
    entry point an RL loop that reads each frame before choosing the next
    action calls);
  - p50 / p99: per-call latency of jx_step with a host sync after each call;
  - e2e: jx_step_host with pinned host buffers (actions in, frames, rewards
    and dones out, every step);
  - plain_one_env_per_launch: 1 env of 16 x 16 rooms, one jx_step per step;
  - cpu_baseline: the FP64 oracle on the host cores (all, and one);
  - uneven, large, serve: bounded runs of the uneven batch, the large-scale
    workload and the serving loop, each with its own numbers.

Prints one JSON line. ``--workload uneven|large|serve`` runs only that
workload at full length. ``--impl reference`` times the FP64 CPU oracle on
the headline workload instead (the method's only other implementation here).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s incl. render (frames/s) at 64x64 RGB"
GRAPH_STEPS = 128  # default rollout buffer slots = steps per rollout launch = launches per CUDA graph
MIN_RING = 4  # rollout buffer slots at least: 4 x 50 MB frames > L2
GRAPH_MIN_STEPS = 128  # the per-step graph leg launches at least this many steps (at most 16 x ring)
SUBMIT_SLACK_CYCLES = 2_000_000  # device-side wait (~1 ms) queued before a timed region's first event
KERNEL_SOURCES = ["paper_2605_19926_gb300/csrc/jx_device.cuh", "paper_2605_19926_gb300/csrc/jx_kernels.cu",
                  "paper_2605_19926_gb300/csrc/jx_internal.h"]
BATCH_KERNEL_SOURCES = ["paper_2605_19926_gb300/csrc/jx_device.cuh", "paper_2605_19926_gb300/csrc/jx_batch_kernels.cu",
                        "paper_2605_19926_gb300/csrc/jx_internal.h"]
# the batched-kernel tiling the large-scale record beside the headline pins
# (the autotuner's choice on that workload: 2 warps per block, 1 ray per lane,
# bit planes from side 128, 16-row blocks, one staging buffer)
LARGE_TILING = "2,1,128,16,1"
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


def recorded_traffic_per_env_step(n_envs: int, path: str = TRAFFIC_FILE, sources=None, tiling=None):
    """DRAM bytes per env-step from the ncu record; None when the record is
    missing, was taken on other kernel code or another batched-kernel tiling,
    or is for another env count without saying that its traffic grows in
    proportion to the env-steps."""
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
    return float(tf["dram_bytes_per_env_step"])


def recorded_traffic(n_envs: int, launch_steps: int, path: str = TRAFFIC_FILE, sources=None, tiling=None):
    """DRAM bytes of one launch of `launch_steps` steps from the ncu record
    (scaled from the captured launch by the env-steps processed), or None."""
    b = recorded_traffic_per_env_step(n_envs, path, sources, tiling)
    return None if b is None else b * n_envs * launch_steps


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


class Plan:
    """Index arithmetic of the headline run, for any --steps / --warmup.

    The action stream holds warmup + steps rows: rows [0, warmup) drive the
    untimed warm-up, rows [warmup, warmup + steps) the timed rollout launches.
    The rollout buffer has `ring` slots; the timed launches cover the steps in
    order, `ring` steps each and a shorter last one. Legs after the timed
    region read the stream at wrapped row indices (modulo its length)."""

    def __init__(self, steps: int, warmup: int, ring_slots: int):
        if steps < 1 or warmup < 0 or ring_slots < 1:
            raise ValueError(f"steps >= 1, warmup >= 0, ring_slots >= 1 (got {steps}, {warmup}, {ring_slots})")
        self.steps, self.warmup = steps, warmup
        self.ring = min(ring_slots, max(steps, MIN_RING))
        self.stream_len = warmup + steps
        self.launches = [(warmup + k * self.ring, min(self.ring, steps - k * self.ring))
                         for k in range(-(-steps // self.ring))]
        self.n_graph = max(1, min(16, -(-GRAPH_MIN_STEPS // self.ring)))

    def warmup_slot(self, s: int) -> int:
        return s % self.ring

    def wrapped(self, first: int, count: int) -> list[int]:
        """Rows first, first + 1, ... of the action stream, wrapped to its length."""
        return [(first + i) % self.stream_len for i in range(count)]

    def graph_rows(self, c: int) -> list[int]:
        """Action rows of the c-th `ring` launches of the per-step graph (it continues the stream after the
        timed steps)."""
        return self.wrapped(self.warmup + self.steps + c * self.ring, self.ring)


def roofline(bytes_total: float, ms: float, peak: float, peak_src: str, **extra) -> dict:
    """HBM roofline of a timed region: algorithmic bytes over the region's time."""
    achieved = bytes_total / (ms / 1e3) / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src}
    out.update(extra)
    return out


def measured_peak() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def percentile(xs, q: float):
    if not len(xs):
        return None
    s = sorted(xs)
    return s[min(len(s) - 1, int(q * len(s)))]


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the GPU works. The median
    SM clock is taken over the samples with the GPU busy (utilisation >= 50%),
    over all samples when none is."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap,utilization.gpu")

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

    @staticmethod
    def summarise(text: str) -> dict | None:
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in text.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            try:
                util = float(parts[9]) if len(parts) > 9 else None
            except ValueError:
                util = None
            reasons = {n for n, v in zip(names, parts[5:9]) if v.lower() == "active"}
            rows.append((sm, mx, util, reasons))
        if not rows:
            return None
        busy = [r for r in rows if r[2] is not None and r[2] >= 50.0]
        use = busy or rows
        reasons = set().union(*(r[3] for r in use))
        return {"sm_mhz": statistics.median(r[0] for r in use), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(busy)}

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return self.summarise(out)


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
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "4096 envs, 32x32 DFS key-door mazes, 64x64 RGB, horizon 500, random actions",
                   "sample_envs": n_envs},
        "cpu_baseline": {"value": value, "unit": "env-steps/s", "cores": used, "kind": "oracle",
                         "sample": f"{n_envs} envs x {args.steps} steps of the workload (frames rendered)"},
        "e2e": {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def tiling_dict(t) -> dict:
    """A launch choice as JSON: all zero means the env's own kernel."""
    names = ("warps_per_block", "cols_per_lane", "bits_min_side", "max_rows_per_block", "staging_buffers")
    d = dict(zip(names, t.as_tuple()))
    d["kernel"] = "env kernel" if not any(t.as_tuple()) else "batched kernel"
    return d


def parse_tiling(jx, text: str):
    """`w,c,b,r[,s]` -> a jx.Tiling (staging buffers default to 1), or None for ''."""
    if not text:
        return None
    t = jx.Tiling()
    vals = [int(v) for v in text.split(",")] + [1]
    (t.warps_per_block, t.cols_per_lane, t.bits_min_side, t.max_rows_per_block, t.staging_buffers) = vals[:5]
    return t


def uneven_bytes_per_env_step(groups: list) -> float:
    """Mean compulsory HBM bytes per env-step of an uneven batch (as for one env group)."""
    tot = sum(g["n_envs"] * algorithmic_bytes_per_env_step(g) for g in groups)
    return tot / sum(g["n_envs"] for g in groups)


class Gpu:
    """The process's device context: rank, world, device, the built library."""

    def __init__(self):
        import torch

        self.torch = torch
        self.rank, self.world, self.local = dist_env()
        if self.world > 1:
            import torch.distributed as dist

            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        torch.cuda.set_device(self.local)
        from paper_2605_19926_gb300 import build

        if self.rank == 0:
            build.build()
        if self.world > 1:
            torch.distributed.barrier()
        from paper_2605_19926_gb300 import jx

        self.jx = jx
        self.dev = torch.device("cuda", self.local)

    def barrier(self):
        if self.world > 1:
            self.torch.distributed.barrier()

    def close(self):
        if self.world > 1:
            self.torch.distributed.destroy_process_group()

    def events(self):
        return (self.torch.cuda.Event(enable_timing=True), self.torch.cuda.Event(enable_timing=True))


def uneven_record(g: Gpu, n_envs: int, slots: int, steps: int, tiling_text: str, tune_trials: int) -> dict | None:
    """Uneven batching: n_envs envs of 16 (map side, frame size) groups in one
    persistent launch per rollout of `slots` steps; fixed tiles against
    autotuned tiles, and the autotuned step sequence replayed as a CUDA graph
    of `slots` single-step launches. Returns rank 0's record."""
    torch, jx = g.torch, g.jx
    from paper_2605_19926_gb300 import inputs

    groups = inputs.uneven_groups(n_envs=n_envs, seed=2 + g.rank)
    envs = [jx.Env(c, g.local) for c in groups]
    pinned = parse_tiling(jx, tiling_text)
    batch = jx.Batch(envs, pinned)
    N, F = batch.n, batch.frame_bytes
    T = slots
    K = max(T, (steps // T) * T)
    acts = torch.from_numpy(inputs.action_stream(7 + g.rank, K + T, N)).to(g.dev)
    frames = torch.empty((T, F), dtype=torch.uint8, device=g.dev)  # T x 0.38 GB > L2
    rewards = torch.empty((T, N), dtype=torch.float32, device=g.dev)
    dones = torch.empty((T, N), dtype=torch.uint8, device=g.dev)
    stream = torch.cuda.Stream(device=g.dev)

    def timed_rollouts() -> tuple[float, int]:
        with torch.cuda.stream(stream):
            batch.reset(frames[0], stream)
            batch.rollout(acts[:T], frames, rewards, dones, stream)  # warm-up
        stream.synchronize()
        n0 = batch.launch_count()
        g.barrier()
        e0, e1 = g.events()
        with torch.cuda.stream(stream):
            torch.cuda._sleep(SUBMIT_SLACK_CYCLES)
            e0.record(stream)
            for c in range(K // T):
                batch.rollout(acts[T + c * T: T + (c + 1) * T], frames, rewards, dones, stream)
            e1.record(stream)
        stream.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), g.world, g.dev), batch.launch_count() - n0

    fixed_ms, _ = timed_rollouts()
    fixed_tiling = batch.tiling
    t_tune = time.perf_counter()
    trials = [] if pinned is not None else batch.autotune(mode=1, steps=T, max_trials=tune_trials, stream=stream)
    tune_s = time.perf_counter() - t_tune
    tuned = batch.tiling
    tuned_ms, launches = timed_rollouts()
    # the same steps as a CUDA graph of T single-step launches, replayed
    graph = batch.capture(acts[T: 2 * T], frames, rewards, dones)
    with torch.cuda.stream(stream):
        batch.reset(frames[0], stream)
        graph.launch(stream)
    stream.synchronize()
    g0, g1 = g.events()
    with torch.cuda.stream(stream):
        torch.cuda._sleep(SUBMIT_SLACK_CYCLES)
        g0.record(stream)
        for c in range(K // T):
            graph.launch(stream)
        g1.record(stream)
    stream.synchronize()
    graph_ms = max_over_ranks(g0.elapsed_time(g1), g.world, g.dev)
    graph.close()
    shape = batch.launch_shape()
    batch.close()
    for e in envs:
        e.close()
    del frames, rewards, dones, acts
    if g.rank != 0:
        return None
    bpes = uneven_bytes_per_env_step(groups)
    peak, peak_src = measured_peak()

    def leg(ms, tiling):
        v = g.world * N * K / (ms / 1e3)
        gbs = N * K * bpes / (ms / 1e3) / 1e9
        return {"value": v, "ms_per_step": ms / K, "achieved_gbs": gbs, "frac": gbs / peak,
                "tiling": tiling_dict(tiling)}

    tuned_leg = leg(tuned_ms, tuned)
    per_es = recorded_traffic_per_env_step(N, TRAFFIC_UNEVEN_FILE, BATCH_KERNEL_SOURCES, tuned.as_tuple())
    return {
        "metric": "env-steps/s incl. render (frames/s), uneven batch", "value": tuned_leg["value"],
        "unit": "env-steps/s", "n_gpus": g.world, "steps": K, "warmup": T, "ms_per_step": tuned_ms / K,
        "higher_is_better": True, "scaling": "weak", "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{N:,} envs per GPU, random-wall rooms p=0.3, map side uniform in {{16,32,64,128}}, "
                               "square RGB frames uniform in {32,64,96,128}, 0-8 sprites, uniform random actions",
                   "groups": len(groups), "n_envs_per_gpu": N, "frame_bytes_per_step": F,
                   "l2": f"frames written to a {T}-slot rollout buffer ({T * F / 1e9:.1f} GB) > L2",
                   "launch": {"grid": shape.grid, "block": shape.block, "smem_bytes": shape.smem,
                              "entry": "jx_batch_rollout", "steps_per_launch": T}},
        "roofline": roofline(N * K * bpes, tuned_ms, peak, peak_src,
                             traffic=None if per_es is None else per_es * N * T,
                             traffic_unit="DRAM bytes per launch (ncu record, scaled by env-steps)",
                             algorithmic_bytes_per_env_step=bpes),
        "fixed_tiles": leg(fixed_ms, fixed_tiling), "autotuned": tuned_leg,
        "autotune": {"trials": len(trials), "seconds": tune_s, "mode": "rollout", "steps_per_trial": T},
        "graph_steps": {"value": g.world * N * K / (graph_ms / 1e3), "ms_per_step": graph_ms / K,
                        "how": f"jx_batch_capture of {T} jx_batch_step launches, replayed"},
        "gpu_launches": launches,
    }


def large_record(g: Gpu, n_envs: int, slots: int, steps: int, tiling_text: str, tune_trials: int) -> dict | None:
    """Large scale: n_envs envs of 128 x 128 mazes with 8 x 8 rooms, 16 sprite
    slots, 128 x 128 RGB frames plus the 4-frame grayscale stack written in the
    same pass, horizon 500, `steps` steps of uniform random actions in rollout
    launches of `slots` steps, from a fresh reset (so a run of >= 500 steps
    crosses the horizon: every env starts its next episode in one launch)."""
    torch, jx = g.torch, g.jx
    from paper_2605_19926_gb300 import inputs

    cfg = shard_config(inputs.large_scale(n_envs), g.rank)
    N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    env = jx.Env(cfg, g.local)
    tuned = None
    if tiling_text:
        env.tiling = parse_tiling(jx, tiling_text)  # the batched kernel with this tiling
    elif tune_trials > 0:
        # the env's own kernel against the batched kernel's tilings, before timing
        tuned = env.autotune(mode=1, steps=slots, max_trials=tune_trials)
    T = slots
    K = max(T, (steps // T) * T)
    acts = torch.from_numpy(inputs.action_stream(cfg["seed"], K, N)).to(g.dev)
    frames = torch.empty((T, N, H, W, 3), dtype=torch.uint8, device=g.dev)
    rewards = torch.empty((K, N), dtype=torch.float32, device=g.dev)
    dones = torch.empty((K, N), dtype=torch.uint8, device=g.dev)
    stream = torch.cuda.Stream(device=g.dev)
    t_reset = time.perf_counter()
    with torch.cuda.stream(stream):
        env.reset(frames[0], stream)
    stream.synchronize()
    reset_s = time.perf_counter() - t_reset
    n0 = env.launch_count()
    g.barrier()
    evs = [g.events() for _ in range(K // T)]
    with torch.cuda.stream(stream):
        torch.cuda._sleep(SUBMIT_SLACK_CYCLES)
        for c in range(K // T):
            evs[c][0].record(stream)
            env.rollout(acts[c * T: (c + 1) * T], frames, rewards[c * T: (c + 1) * T], dones[c * T: (c + 1) * T],
                        stream)
            evs[c][1].record(stream)
    stream.synchronize()
    per_launch = [a.elapsed_time(b) for a, b in evs]
    ms = max_over_ranks(evs[0][0].elapsed_time(evs[-1][1]), g.world, g.dev)
    launches = env.launch_count() - n0
    done_steps = dones.sum(dim=1).cpu().numpy()
    shape = env.launch_shape()
    tiling = env.tiling
    env.close()
    del frames, rewards, dones, acts
    if g.rank != 0:
        return None
    gray = H * W  # one plane per env-step (all four at an episode start)
    bpes = algorithmic_bytes_per_env_step(cfg) + gray
    peak, peak_src = measured_peak()
    # launches whose steps end episodes (the horizon), against the others
    ends = [int(done_steps[c * T: (c + 1) * T].sum()) for c in range(K // T)]
    normal = [per_launch[c] for c in range(1, K // T) if ends[c] == 0]
    per_es = recorded_traffic_per_env_step(N, TRAFFIC_LARGE_FILE, BATCH_KERNEL_SOURCES, tiling.as_tuple())
    return {
        "metric": "env-steps/s incl. render (frames/s), 128x128 RGB + gray stack",
        "value": g.world * N * K / (ms / 1e3), "unit": "env-steps/s", "n_gpus": g.world, "steps": K, "warmup": 0,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{N} envs per GPU, 128x128 DFS mazes with 8x8 open rooms, 16 sprite slots (key, goal, "
                               "0-14 distractors), 128x128 RGB + 4-frame grayscale stack in the same pass, horizon 500, "
                               "uniform random actions, from a fresh reset",
                   "l2": f"frames written to a {T}-slot rollout buffer ({T * N * H * W * 3 / 1e9:.1f} GB) > L2",
                   "launch": {"grid": shape.grid, "block": shape.block, "smem_bytes": shape.smem,
                              "entry": "jx_rollout", "steps_per_launch": T}},
        "roofline": roofline(N * K * bpes, ms, peak, peak_src,
                             traffic=None if per_es is None else per_es * N * T,
                             traffic_unit="DRAM bytes per launch (ncu record, scaled by env-steps)",
                             algorithmic_bytes_per_env_step=bpes),
        "reset_seconds": reset_s,
        "episode_ends": sum(ends),
        "launch_ms": {"median_normal": statistics.median(normal) if normal else None,
                      "first": per_launch[0],
                      "horizon_launches": [{"launch": c, "ms": per_launch[c], "episode_ends": ends[c]}
                                           for c in range(K // T) if ends[c] > 0]},
        "tiling": tiling_dict(tiling),
        "autotune_trials": len(tuned) if tuned else 0,
        "gpu_launches": launches,
    }


def serve_record(g: Gpu, actors: int, duration: float, session_steps: int, budget_gb: float) -> dict | None:
    """Serving: `actors` actor groups submit step requests with Poisson
    arrivals (mean gap 2 ms) to the continuous-batching server for `duration`
    seconds. Each group runs sessions of `session_steps` requests; a session's
    batch is log-uniform in [16, 4096] envs of 32x32 or 64x64 key-door mazes,
    64x64 RGB. Sessions are admitted under a `budget_gb` state+frame budget.
    Reports p50 / p99 request latency (submit to completion) and aggregate
    env-steps/s over the window after a warm-up."""
    import concurrent.futures as cf
    import heapq

    jx = g.jx
    from paper_2605_19926_gb300 import inputs

    seed = 3 + g.rank
    warm = min(2.0, duration / 4)
    server = jx.Server(budget_bytes=int(budget_gb * 1e9), max_sessions=4 * actors, max_inflight=4,
                       max_map_side=64, device=g.local)
    pool = cf.ThreadPoolExecutor(max_workers=4)
    session = [None] * actors  # open Session or None
    opening = [None] * actors  # future of a pending open
    left = [0] * actors
    k_next = [0] * actors
    acts = [None] * actors
    gaps = [inputs.arrival_gaps(seed, a, 1 << 16) for a in range(actors)]
    gi = [1] * actors
    heap = [(float(gaps[a][0]), a) for a in range(actors)]
    heapq.heapify(heap)
    t0 = time.perf_counter()
    stats_mark = None
    submitted = 0
    act_bytes = 0
    while heap:
        t_rel, a = heapq.heappop(heap)
        if t_rel > duration:
            break
        while time.perf_counter() - t0 < t_rel:
            pass
        if stats_mark is None and t_rel >= warm:
            server.latencies()  # drop the warm-up requests
            stats_mark = (time.perf_counter(), server.stats(), submitted, act_bytes)
        if session[a] is None and opening[a] is not None and opening[a].done():
            session[a] = opening[a].result()
            opening[a] = None
            if session[a] is not None:
                left[a] = session_steps
                n = session[a].n
                acts[a] = np.random.default_rng([seed, a, k_next[a]]).integers(0, 7, size=(8, n), dtype=np.uint8)
        if session[a] is not None:
            session[a].submit(acts[a][left[a] % 8])
            submitted += 1
            act_bytes += session[a].n
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
    t_stats0, st0, sub0, ab0 = stats_mark
    window = t_end - t_stats0
    env_steps = st_end["env_steps"] - st0["env_steps"]
    reqs = st_end["requests_done"] - st0["requests_done"]
    launches = st_end["launches"] - st0["launches"]
    groups = st_end["groups_launched"] - st0["groups_launched"]
    server.close()
    value = env_steps / window
    tot = max_over_ranks(window * 1e3, g.world, g.dev)
    if g.rank != 0:
        return None
    return {
        "metric": "env-steps/s incl. render (frames/s), served requests", "value": value * g.world,
        "unit": "env-steps/s", "n_gpus": g.world, "requests": int(reqs),
        "ms_per_request": tot / max(1, reqs), "higher_is_better": True, "scaling": "weak", "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{actors} actor groups, Poisson arrivals (mean gap 2 ms), sessions of "
                               f"{session_steps} requests, batch log-uniform in [16, 4096] envs, 32x32 or 64x64 "
                               "key-door mazes, 64x64 RGB, continuous batching",
                   "budget_gb": budget_gb, "seconds": duration, "measured_seconds": window,
                   "max_inflight_launches": 4},
        "p50_step_ms": float(np.percentile(lat, 50)) * 1e3 if len(lat) else None,
        "p99_step_ms": float(np.percentile(lat, 99)) * 1e3 if len(lat) else None,
        "latency_samples": int(len(lat)),
        "requests_per_s": reqs / window, "submitted_per_s": (submitted - sub0) / window,
        "mean_sessions_per_launch": groups / max(1, launches), "launches": int(launches),
        "mean_envs_per_request": env_steps / max(1, reqs),
        "server": {k: st_end[k] for k in ("peak_bytes_in_use", "budget_bytes", "peak_sessions",
                                          "peak_inflight_launches", "rejected_opens")},
        "roofline": None,
        "roofline_note": "latency-bound: the offered load is far below the HBM roofline",
        "e2e": {"value": value * g.world, "unit": "env-steps/s",
                "h2d_bytes_per_request": (act_bytes - ab0) / max(1, submitted - sub0), "d2h_bytes_per_request": 0,
                "how": "host actions submitted per request through jx_server_submit; results stay on the device"},
        "gpu_launches": int(launches),
    }


def headline(g: Gpu, args) -> dict | None:
    """The headline workload (4096 key-door mazes, 64 x 64) and the legs beside it."""
    torch, jx = g.torch, g.jx
    from paper_2605_19926_gb300 import inputs

    base_cfg = inputs.batched_keydoor_mazes(args.n_envs)
    cfg = shard_config(base_cfg, g.rank)
    N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    plan = Plan(args.steps, args.warmup, args.ring_slots)
    ring = plan.ring
    env = jx.Env(cfg, g.local)
    tuned = None
    if not args.no_autotune:
        # the env's own kernel against the batched kernel's tilings, before timing
        tuned = env.autotune(mode=1, steps=ring, max_trials=args.tune_trials)
    # inputs resident in HBM before timing: the whole action stream
    acts_host = inputs.action_stream(cfg["seed"], plan.stream_len, N)
    acts = torch.from_numpy(acts_host).to(g.dev)
    # the single-step leg's actions: its own row for each of its launches
    n_step_graph = plan.n_graph * ring
    step_acts = torch.cat([acts.index_select(0, torch.tensor(plan.graph_rows(c), device=g.dev))
                           for c in range(plan.n_graph)])
    frames = torch.zeros((ring, N, H, W, 3), dtype=torch.uint8, device=g.dev)  # 6.4 GB at 128 slots
    rewards = torch.empty((ring, N), dtype=torch.float32, device=g.dev)
    dones = torch.empty((ring, N), dtype=torch.uint8, device=g.dev)
    stream = torch.cuda.Stream(device=g.dev)
    torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        env.reset(frames[0], stream)
        for s in range(plan.warmup):
            k = plan.warmup_slot(s)
            env.step(acts[s], frames[k], rewards[k], dones[k], stream)
    stream.synchronize()

    # single-step entry point: a CUDA graph of n_step_graph jx_step launches
    # (frames into the rollout buffer's slots in turn)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        for i in range(n_step_graph):
            k = i % ring
            env.step(step_acts[i], frames[k], rewards[k], dones[k], torch.cuda.current_stream())
    torch.cuda.synchronize()
    # the capture itself ran nothing; the env state is still after the warm-up

    # timed region: the steps in rollout launches of at most `ring` steps
    launches_before = env.launch_count()
    g.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = g.events()
    with torch.cuda.stream(stream):
        # a ~1 ms device-side wait ahead of the first event keeps the host's
        # submission of the launches out of the timed region (device time only)
        torch.cuda._sleep(SUBMIT_SLACK_CYCLES)
        ev0.record(stream)
        for start, n in plan.launches:
            env.rollout(acts[start: start + n], frames[:n], rewards[:n], dones[:n], stream)
        ev1.record(stream)
    stream.synchronize()
    ms = ev0.elapsed_time(ev1)
    gpu_launches = env.launch_count() - launches_before
    t_max = max_over_ranks(ms, g.world, g.dev)
    g.barrier()
    value = job_value(g.world, N, args.steps, t_max)

    # the single-step entry point on the same workload: the graph replayed
    # once untimed (its first launch uploads it), then once timed
    torch.cuda.synchronize()
    g0, g1 = g.events()
    with torch.cuda.stream(stream):
        graph.replay()
        torch.cuda._sleep(SUBMIT_SLACK_CYCLES)
        g0.record(stream)
        graph.replay()
        g1.record(stream)
    stream.synchronize()
    step_ms = g0.elapsed_time(g1) / n_step_graph

    # per-step latency (eager launch + kernel, one step at a time)
    lat = []
    with torch.cuda.stream(stream):
        for i, row in enumerate(plan.wrapped(plan.warmup, args.latency_steps)):
            a, b = g.events()
            a.record(stream)
            k = i % ring
            env.step(acts[row], frames[k], rewards[k], dones[k], stream)
            b.record(stream)
            b.synchronize()
            lat.append(a.elapsed_time(b))

    # the plain method: one environment, one jx_step launch per step (16 x 16 rooms)
    plain = None
    if g.rank == 0 and args.plain_steps > 0:
        pc = inputs.single_env_rooms()
        penv = jx.Env(pc, g.local)
        pa = torch.from_numpy(inputs.action_stream(pc["seed"], args.plain_steps, 1)).to(g.dev)
        pf = torch.empty((1, pc["frame_h"], pc["frame_w"], 3), dtype=torch.uint8, device=g.dev)
        pr = torch.empty(1, dtype=torch.float32, device=g.dev)
        pd = torch.empty(1, dtype=torch.uint8, device=g.dev)
        with torch.cuda.stream(stream):
            penv.reset(pf, stream)
            for i in range(min(8, args.plain_steps)):
                penv.step(pa[i], pf, pr, pd, stream)
            p0, p1 = g.events()
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
                a, b = g.events()
                a.record(stream)
                penv.step(pa[i], pf, pr, pd, stream)
                b.record(stream)
                b.synchronize()
                plat.append(a.elapsed_time(b))
        plain = {"value": args.plain_steps / (pms / 1e3), "unit": "env-steps/s", "ms_per_step": pms / args.plain_steps,
                 "p50_step_ms": percentile(plat, 0.5), "p99_step_ms": percentile(plat, 0.99),
                 "workload": f"1 env, 16x16 random rooms (p = 0.25), 64x64 RGB, {args.plain_steps} uniform random steps, "
                             "one jx_step launch per step"}
        penv.close()

    # end to end through the public host-buffer entry point (pinned host memory)
    h_act = torch.empty(N, dtype=torch.uint8).pin_memory()
    h_frames = torch.empty((N, H, W, 3), dtype=torch.uint8).pin_memory()
    h_rew = torch.empty(N, dtype=torch.float32).pin_memory()
    h_done = torch.empty(N, dtype=torch.uint8).pin_memory()
    rows = plan.wrapped(plan.warmup, args.e2e_steps + 3)
    for i in range(3):
        h_act.numpy()[:] = acts_host[rows[i]]
        env.step_host(h_act, h_frames, h_rew, h_done, stream)
    t0 = time.perf_counter()
    for i in range(args.e2e_steps):
        h_act.numpy()[:] = acts_host[rows[3 + i]]
        env.step_host(h_act, h_frames, h_rew, h_done, stream)
    e2e_s = time.perf_counter() - t0
    e2e_value = g.world * N * args.e2e_steps / e2e_s  # every rank runs the same count; host clock per rank

    shape, chunk = env.rollout_shape(ring)  # the timed launches
    step_shape = env.launch_shape()
    tiling = env.tiling
    graph.reset()
    env.close()
    del frames, rewards, dones, acts, step_acts
    torch.cuda.empty_cache()
    if g.rank != 0:
        return None

    peak, peak_src = measured_peak()
    bytes_total = sum(rollout_bytes(cfg, N, n) for _, n in plan.launches)
    per_es = recorded_traffic_per_env_step(N)
    traffic = None if per_es is None else per_es * N * args.steps / len(plan.launches)
    step_bytes = algorithmic_bytes_per_env_step(cfg) * N
    cpu = None
    if not args.no_cpu_baseline and g.world == 1:
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
    return {
        "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": g.world, "steps": args.steps,
        "warmup": plan.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "4096 envs per GPU, 32x32 random DFS key-door mazes, 64x64 RGB uint8, horizon 500, "
                               "auto-reset, uniform random actions, seed 1",
                   "n_envs_per_gpu": N, "map_side": cfg["map_side"], "frame": f"{H}x{W}x3 uint8",
                   "parallelism": f"replicas x{g.world}",
                   "l2": f"frames written to a {ring}-slot rollout buffer ({ring * N * H * W * 3 / 1e9:.2f} GB) > L2",
                   "launch": {"grid": shape.grid, "block": shape.block, "smem_bytes": shape.smem,
                              "entry": "jx_rollout", "steps_per_launch": ring, "handoff_chunk_steps": chunk,
                              "timed_launches": len(plan.launches), "step_grid": step_shape.grid,
                              "tiling": tiling_dict(tiling), "autotune_trials": len(tuned) if tuned else 0}},
        "p50_step_ms": percentile(lat, 0.5), "p99_step_ms": percentile(lat, 0.99),
        "latency": {"how": "jx_step launched alone, host sync after each call, CUDA events around the launch",
                    "samples": len(lat)},
        "per_step_launch": {"value": g.world * N / (step_ms / 1e3), "unit": "env-steps/s", "ms_per_step": step_ms,
                            "roofline": roofline(step_bytes, step_ms, peak, peak_src,
                                                 algorithmic_bytes_per_launch=step_bytes),
                            "how": f"jx_step, CUDA graph of {n_step_graph} launches (each its own action row), "
                                   "one timed replay after an untimed one"},
        "plain_one_env_per_launch": plain,
        "roofline": roofline(bytes_total, t_max, peak, peak_src, traffic=traffic,
                             traffic_unit="DRAM bytes per launch (ncu record, scaled by env-steps)",
                             algorithmic_bytes_per_step=bytes_total / args.steps,
                             algorithmic_bytes_per_launch=bytes_total / len(plan.launches),
                             kernel="jx_rollout (env kernel, or the batched kernel when autotuned to it)"),
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "env-steps/s", "h2d_bytes_per_step": N,
                "d2h_bytes_per_step": N * H * W * 3 + 4 * N + N,
                "how": f"jx_step_host, pinned host buffers, {args.e2e_steps} steps, host clock"},
        "gpu_launches": gpu_launches,
    }


def extras(g: Gpu, args) -> dict:
    """Bounded runs of the uneven batch, the large-scale workload and the
    serving loop beside the headline (each failure is recorded, not raised)."""
    out = {}
    runs = {
        "uneven": lambda: uneven_record(g, args.uneven_envs, args.uneven_slots, args.extra_uneven_steps, args.tiling,
                                        args.tune_trials),
        "large": lambda: large_record(g, args.large_envs, args.large_slots, args.extra_large_steps,
                                      args.large_tiling, 0),
        "serve": lambda: serve_record(g, args.actors, args.extra_serve_seconds, args.session_steps, args.budget_gb),
    }
    for name, fn in runs.items():
        t0 = time.perf_counter()
        try:
            rec = fn()
        except Exception as exc:  # recorded in the line: the headline still prints
            rec = {"error": f"{type(exc).__name__}: {exc}"}
        if rec is not None:
            rec["wall_seconds"] = time.perf_counter() - t0
        out[name] = rec
        g.torch.cuda.empty_cache()
    return out


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
    ap.add_argument("--no-extras", action="store_true", help="headline only: skip the uneven / large / serve records")
    ap.add_argument("--plain-steps", type=int, default=1000)
    ap.add_argument("--ring-slots", type=int, default=GRAPH_STEPS,
                    help="rollout buffer slots = steps per rollout launch = launches per CUDA graph")
    ap.add_argument("--workload", default="mazes", choices=["mazes", "uneven", "serve", "large"],
                    help="mazes: 4096 key-door mazes (the headline, with bounded uneven / large / serve records); "
                         "uneven, large, serve: only that workload, at full length")
    ap.add_argument("--actors", type=int, default=64)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--extra-serve-seconds", type=float, default=10.0)
    ap.add_argument("--session-steps", type=int, default=250)
    ap.add_argument("--budget-gb", type=float, default=40.0)
    ap.add_argument("--large-envs", type=int, default=65536)
    ap.add_argument("--large-slots", type=int, default=8, help="steps per rollout launch of the large workload")
    ap.add_argument("--extra-large-steps", type=int, default=512, help="large record beside the headline: steps")
    ap.add_argument("--large-tiling", default=LARGE_TILING,
                    help="large record beside the headline: batched-kernel tiling w,c,b,r[,s] ('' = env kernel)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip jx_autotune before timing (the env's own kernel with its fixed tiles)")
    ap.add_argument("--uneven-slots", type=int, default=16, help="steps per rollout launch of the uneven batch")
    ap.add_argument("--uneven-envs", type=int, default=16384)
    ap.add_argument("--extra-uneven-steps", type=int, default=128, help="uneven record beside the headline: steps")
    ap.add_argument("--tiling", default="",
                    help="uneven batch and large scale: w,c,b,r[,s] batched-kernel tiling to use instead of autotuning")
    ap.add_argument("--tune-trials", type=int, default=1000)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    default_steps = args.steps == ap.get_default("steps")
    if args.impl == "reference":
        from paper_2605_19926_gb300 import inputs

        run_reference(args, inputs.batched_keydoor_mazes(args.n_envs))
        return

    g = Gpu()
    clocks = ClockSampler(g.local)
    clocks.start()
    time.sleep(0.3)
    window = "the whole run"
    if args.workload == "uneven":
        line = uneven_record(g, args.uneven_envs, args.uneven_slots, 512 if default_steps else args.steps,
                             args.tiling, args.tune_trials)
    elif args.workload == "large":
        line = large_record(g, args.large_envs, args.large_slots, 1000 if default_steps else args.steps, args.tiling,
                            0 if args.no_autotune else args.tune_trials)
    elif args.workload == "serve":
        line = serve_record(g, args.actors, args.serve_seconds, args.session_steps, args.budget_gb)
    else:
        line = headline(g, args)
        window = "the headline's timed region, its legs and the uneven / large / serve records"
        if line is not None and g.world == 1 and not args.no_extras:
            line.update(extras(g, args))
    clk = clocks.stop()
    if line is not None:
        if clk is not None:
            clk["window"] = window
        line["clocks"] = clk
        print(json.dumps(line), flush=True)
    g.close()


if __name__ == "__main__":
    main()
