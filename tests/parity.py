"""Lockstep parity harness: the CUDA path (through the C ABI) against the oracle.

Tolerances (from the accuracy rules the hot path is held to):
- bit-exact: rewards (float32), done flags, key/door state, episode counters,
  generated maps, spawn cells and object cells; hit cell and hit side of every
  ray;
- pose within 1e-5 absolute; perpendicular distance within 1e-5 relative;
- pixels: at most 1e-4 of all pixels may differ, and only pixels the oracle
  flags as lying on an edge that finite precision can move (slice edges whose
  height rounding is within tolerance, sprite silhouette edges).

Where finite precision admits more than one correct result, the GPU's result
must be one of them, and nothing is skipped:
- a corner ray (a DDA tie within 1e-5 cells, or a hit within 1e-5 of a grid
  corner) must hit the cell and side of the oracle's cast with its ties taken
  towards x or towards y, and its column must match the frame of that choice;
  corner rays are counted and must stay <= 0.1% of rays;
- a near-tie step (a collision or pickup decision within 1e-5 cells of
  flipping) must equal the oracle's step with those decisions taken one of
  the ways they admit (rewards, done, keys, counters exact, pose within 1e-5);
  near ties are counted per run (consecutive checked steps of one env in one
  episode) and the runs must stay <= 0.1% of env-steps.
"""

from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np
import torch

import oracle
from paper_2605_19926_gb300 import inputs, jx

TOL_POSE = 1e-5
TOL_PERP_REL = 1e-5
PIXEL_FRAC = 1e-4
CORNER_FRAC = 1e-3
# Near-tie steps are checked against every outcome the tie admits and counted
# per run: an agent whose box edge ends within 1e-5 of a wall face stays in the
# tie for every step it keeps pushing into that wall, one run of steps.
NEAR_TIE_FRAC = 1e-3
NTHREADS = max(1, min(16, os.cpu_count() or 1))
# the decisions a near tie admits: (collision x, collision y, pickup x, pickup y) biases
TIE_VARIANTS = [(cx, cy, px, py) for cx in (1, -1) for cy in (1, -1) for px in (1, -1) for py in (1, -1)]


def oracle_cfg(cfg: dict) -> np.ndarray:
    return oracle.make_config(**cfg)


def to_oracle(env: jx.Env, blob: np.ndarray, idx=None) -> np.ndarray:
    """Decode the GPU state blob into oracle env records (exactly)."""
    f = env.fields(blob)
    N, S, K = env.n, env.S, env.K
    idx = np.arange(N) if idx is None else np.asarray(idx)
    o = np.zeros(len(idx), oracle.ENV_DTYPE)
    o["x"] = f["cell_x"][idx].astype(np.float64) + f["frac_x"][idx].astype(np.float64)
    o["y"] = f["cell_y"][idx].astype(np.float64) + f["frac_y"][idx].astype(np.float64)
    o["theta0"] = f["theta0"][idx].astype(np.float64)
    o["turn"] = f["turn"][idx]
    o["t"] = f["t"][idx]
    o["episode"] = f["episode"][idx]
    o["keys"] = f["flags"][idx] & 7
    obj = f["obj"][idx].astype(np.int32)
    for k, name in enumerate(("key_x", "key_y", "goal_x", "goal_y", "door_x", "door_y")):
        o[name] = obj[:, k]
    o["n_sprites"] = f["nspr"][idx]
    if K:
        o["spr_x"][:, :K] = f["spr_x"][idx]
        o["spr_y"][:, :K] = f["spr_y"][idx]
        o["spr_type"][:, :K] = f["spr_type"][idx]
    o["map"][:, : S * S] = f["map"][idx].reshape(len(idx), S * S)
    return o


@dataclass
class Stats:
    pixels: int = 0
    pixel_mismatch: int = 0
    rays: int = 0
    corner_rays: int = 0
    corner_rays_other_way: int = 0  # corner rays the GPU took the other way from the exact FP64 cast
    env_steps: int = 0
    near_ties: int = 0  # near-tie env-steps (each checked against the outcomes it admits)
    near_tie_runs: int = 0
    near_ties_other_way: int = 0  # near-tie steps whose GPU outcome differs from the exact FP64 step
    key_events: int = 0
    goal_events: int = 0
    resets: int = 0
    notes: list = field(default_factory=list)
    _tie_last: dict = field(default_factory=dict, repr=False)

    def tie(self, key, episode: int, step: int, step_gap: int):
        """Count a near-tie env-step; a new run unless the same env's previous
        checked step (same episode) was one too."""
        self.near_ties += 1
        if self._tie_last.get(key) != (episode, step - step_gap):
            self.near_tie_runs += 1
        self._tie_last[key] = (episode, step)

    def check(self):
        assert self.pixel_mismatch <= PIXEL_FRAC * max(self.pixels, 1), self
        assert self.corner_rays <= CORNER_FRAC * max(self.rays, 1), self
        assert self.near_tie_runs <= max(1, NEAR_TIE_FRAC * self.env_steps), self


def compare_generated(gpu: np.ndarray, ref: np.ndarray, S: int, K: int, where: str = ""):
    """A freshly generated episode: everything exact (theta0 is the float32 rounding of the FP64 value)."""
    n = S * S
    assert (gpu["map"][:, :n] == ref["map"][:, :n]).all(), f"maps differ {where}"
    for name in ("key_x", "key_y", "goal_x", "goal_y", "door_x", "door_y", "n_sprites", "turn", "t", "episode",
                 "keys"):
        assert (gpu[name] == ref[name]).all(), f"{name} differs {where}"
    assert (gpu["x"] == ref["x"]).all() and (gpu["y"] == ref["y"]).all(), f"spawn differs {where}"
    assert (gpu["theta0"].astype(np.float32) == ref["theta0"].astype(np.float32)).all(), f"theta0 differs {where}"
    if K:
        assert (gpu["spr_type"][:, :K] == ref["spr_type"][:, :K]).all()
        assert (gpu["spr_x"][:, :K] == ref["spr_x"][:, :K].astype(np.float32)).all()
        assert (gpu["spr_y"][:, :K] == ref["spr_y"][:, :K].astype(np.float32)).all()


def render_ref(ocfg: np.ndarray, states: np.ndarray) -> dict:
    """The oracle's frames, rays and ambiguity flags of `states`, plus, for the
    envs that have a corner ray, the frames with every tie taken towards x
    (+1) and towards y (-1): the results a corner ray admits."""
    states = np.ascontiguousarray(states)
    ref = oracle.render(ocfg, states, nthreads=NTHREADS)
    ec = np.nonzero(ref["rays"]["corner"].any(axis=1))[0]
    ref["variants"] = {"envs": ec}
    if len(ec):
        for b in (1, -1):
            ref["variants"][b] = oracle.render(ocfg, states[ec], nthreads=NTHREADS, bias=b)
    return ref


def _variant_rows(ref: dict, e: int):
    """Row of env e in the biased renders."""
    ec = ref["variants"]["envs"]
    k = int(np.searchsorted(ec, e))
    assert k < len(ec) and ec[k] == e
    return k


def compare_frames(gpu_frames: np.ndarray, ref: dict, stats: Stats):
    """Every pixel equals the oracle's, except where the oracle flags an edge
    that finite precision can move; a corner-ray column must equal the column
    of the oracle frame with that ray's tie taken one of its two ways."""
    of, amb = ref["frames"].copy(), ref["ambiguous"].astype(bool)
    corner = ref["rays"]["corner"].astype(bool)
    for e, c in np.argwhere(corner):
        k = _variant_rows(ref, e)
        for b in (1, -1):
            v = ref["variants"][b]
            vamb = v["ambiguous"][k, :, c].astype(bool)
            if ((gpu_frames[e, :, c] == v["frames"][k, :, c]).all(axis=-1) | vamb).all():
                of[e, :, c] = v["frames"][k, :, c]
                amb[e, :, c] = vamb
                break
        else:
            raise AssertionError(f"corner column ({e}, {c}) matches neither tie decision")
    mism = (gpu_frames != of).any(axis=-1)
    bad = mism & ~amb
    if bad.any():
        e, y, x = np.argwhere(bad)[0]
        raise AssertionError(f"pixel ({e},{y},{x}) gpu {gpu_frames[e, y, x]} oracle {of[e, y, x]} not an edge")
    stats.pixels += mism.size
    stats.pixel_mismatch += int(mism.sum())


def _perp_ok(po: np.ndarray, pg: np.ndarray) -> np.ndarray:
    pg = pg.astype(np.float64)
    diff = np.where(po == pg, 0.0, np.abs(pg - po))
    rel = np.where(po > 0, diff / np.where(po > 0, po, 1.0), diff)
    return rel <= TOL_PERP_REL


def compare_rays(hits: np.ndarray, perp: np.ndarray, ref: dict, stats: Stats):
    """Hit cell and side exact, perp within 1e-5 relative, slice height exact
    unless its rounding is within tolerance; a corner ray must equal the
    oracle's cast with its tie taken towards x or towards y."""
    rays = ref["rays"]
    corner = rays["corner"].astype(bool)
    ok = ~corner
    assert (hits[..., 0][ok] == rays["cell_x"][ok]).all(), "hit cell x"
    assert (hits[..., 1][ok] == rays["cell_y"][ok]).all(), "hit cell y"
    assert (hits[..., 2][ok] == rays["side"][ok]).all(), "hit side"
    assert _perp_ok(rays["perp"][ok], perp[ok]).all(), "perp relative error"
    hok = ok & ~rays["h_ambiguous"].astype(bool)
    assert (hits[..., 3][hok] == rays["h"][hok]).all(), "slice height"
    for e, c in np.argwhere(corner):
        k = _variant_rows(ref, e)
        for b in (1, -1):
            r = ref["variants"][b]["rays"][k, c]
            if (hits[e, c, 0], hits[e, c, 1], hits[e, c, 2]) != (r["cell_x"], r["cell_y"], r["side"]):
                continue
            assert _perp_ok(np.array([r["perp"]]), np.array([perp[e, c]])).all(), f"corner ray ({e}, {c}) perp"
            assert r["h_ambiguous"] or hits[e, c, 3] == r["h"], f"corner ray ({e}, {c}) slice height"
            if (r["cell_x"], r["cell_y"], r["side"]) != (rays["cell_x"][e, c], rays["cell_y"][e, c], rays["side"][e, c]):
                stats.corner_rays_other_way += 1
            break
        else:
            raise AssertionError(f"corner ray ({e}, {c}) hit {tuple(hits[e, c, :3])} matches neither tie decision")
    stats.rays += corner.size
    stats.corner_rays += int(corner.sum())


class Run:
    """One CUDA env batch plus its torch output buffers."""

    def __init__(self, cfg: dict, device: int = 0):
        self.cfg = cfg
        self.env = jx.Env(cfg, device)
        self.ocfg = oracle_cfg(cfg)
        N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
        dev = torch.device("cuda", device)
        self.frames = torch.zeros((N, H, W, 3), dtype=torch.uint8, device=dev)
        self.rewards = torch.zeros(N, dtype=torch.float32, device=dev)
        self.dones = torch.zeros(N, dtype=torch.uint8, device=dev)
        self.hits = torch.zeros((N, W, 4), dtype=torch.int32, device=dev)
        self.perp = torch.zeros((N, W), dtype=torch.float32, device=dev)
        self.actions = torch.zeros(N, dtype=torch.uint8, device=dev)
        self.dev = dev
        self.gray = GrayModel(N, H, W) if cfg.get("gray_stack") else None

    def state(self, idx=None) -> np.ndarray:
        return to_oracle(self.env, self.env.get_state(), idx)

    def rays(self):
        self.env.debug_rays(self.hits, self.perp)
        torch.cuda.synchronize()
        return self.hits.cpu().numpy(), self.perp.cpu().numpy()

    def reset(self):
        self.env.reset(self.frames)
        torch.cuda.synchronize()

    def step(self, actions: np.ndarray):
        self.actions.copy_(torch.from_numpy(actions))
        self.env.step(self.actions, self.frames, self.rewards, self.dones)
        torch.cuda.synchronize()
        return self.frames.cpu().numpy(), self.rewards.cpu().numpy(), self.dones.cpu().numpy()


class GrayModel:
    """The grayscale stack a Run's envs should hold, rebuilt on the host from the
    GPU's RGB frames and step counters: the frame of episode step t in plane
    t mod 4, an episode's first frame in all four planes."""

    def __init__(self, n: int, H: int, W: int):
        self.planes = np.zeros((n, 4, H, W), np.uint8)

    def update(self, frames: np.ndarray, t: np.ndarray):
        g = oracle.gray(frames)
        for e in range(len(t)):
            if t[e] == 0:
                self.planes[e, :] = g[e]
            else:
                self.planes[e, t[e] % 4] = g[e]

    def check(self, env: jx.Env, idx=None):
        f = env.fields(env.get_state())
        got = f["gray"] if idx is None else f["gray"][idx]
        want = self.planes if idx is None else self.planes[idx]
        assert (got == want).all(), "grayscale stack differs"


def check_reset(run: Run, stats: Stats, idx=None):
    N = run.cfg["n_envs"]
    idx = np.arange(N) if idx is None else np.asarray(idx)
    run.reset()
    if run.gray is not None:
        run.gray.update(run.frames.cpu().numpy(), run.env.fields(run.env.get_state())["t"])
        run.gray.check(run.env)
    gpu = run.state(idx)
    ref = oracle.generate(run.ocfg, idx.astype(np.int32), 0, nthreads=NTHREADS)
    compare_generated(gpu, ref, run.env.S, run.env.K, "at reset")
    # render parity on the exact same state (the GPU's, decoded)
    out = render_ref(run.ocfg, gpu)
    compare_frames(run.frames.cpu().numpy()[idx], out, stats)
    hits, perp = run.rays()
    compare_rays(hits[idx], perp[idx], out, stats)


def forward_biased_actions(seed: int, step: int, n: int) -> np.ndarray:
    """60% forward, otherwise a turn or a strafe: a walk that travels far enough
    to reach keys, doors and goals within a short test."""
    rng = np.random.default_rng([seed, step, 77])
    other = rng.choice(np.array([3, 4, 5, 6], np.uint8), size=n)
    return np.where(rng.random(n) < 0.6, np.uint8(1), other).astype(np.uint8)


def _same_state(g: np.ndarray, r: np.ndarray, done: bool, S: int, K: int) -> bool:
    """One env record of the GPU equals the oracle's after a step: a fresh
    episode exactly (done), else counters, keys and map exactly and the pose
    within TOL_POSE."""
    n = S * S
    if not (g["map"][:n] == r["map"][:n]).all():
        return False
    if any(g[k] != r[k] for k in ("turn", "t", "episode", "keys")):
        return False
    if done:
        return (all(g[k] == r[k] for k in ("x", "y", "key_x", "key_y", "goal_x", "goal_y", "door_x", "door_y",
                                           "n_sprites"))
                and np.float32(g["theta0"]) == np.float32(r["theta0"])
                and (g["spr_type"][:K] == r["spr_type"][:K]).all())
    return abs(g["x"] - r["x"]) <= TOL_POSE and abs(g["y"] - r["y"]) <= TOL_POSE


def check_step(ocfg: np.ndarray, idx: np.ndarray, pre: np.ndarray, actions: np.ndarray, cur: np.ndarray,
               rewards: np.ndarray, dones: np.ndarray, S: int, K: int, stats: Stats, step: int, where: str = "",
               key=(), step_gap: int = 1):
    """Step the oracle from `pre` (the GPU's pre-step states of envs idx) and
    compare with the GPU's rewards, dones and post-step states `cur`. A
    near-tie step must equal the oracle's step under one of the decisions the
    tie admits."""
    idx = np.asarray(idx, dtype=np.int32)
    ref_st = np.ascontiguousarray(pre).copy()
    ref = oracle.step(ocfg, idx, ref_st, actions, nthreads=NTHREADS)
    ev = ref["events"]
    near = (ev & oracle.EV_NEAR_TIE) != 0
    ok = ~near
    stats.env_steps += len(idx)
    stats.key_events += int(((ev & oracle.EV_KEY) != 0)[ok].sum())
    stats.goal_events += int(((ev & oracle.EV_GOAL) != 0)[ok].sum())
    assert (rewards[ok] == ref["rewards"][ok]).all(), f"rewards differ at step {step} {where}"
    assert (dones[ok] == ref["dones"][ok]).all(), f"dones differ at step {step} {where}"
    done = (ref["dones"] == 1) & ok
    stats.resets += int(done.sum())
    if done.any():
        compare_generated(cur[done], ref_st[done], S, K, f"after auto-reset at step {step} {where}")
    live = ok & ~done
    for name in ("turn", "t", "episode", "keys"):
        assert (cur[name][live] == ref_st[name][live]).all(), f"{name} differs at step {step} {where}"
    assert (cur["map"][live][:, : S * S] == ref_st["map"][live][:, : S * S]).all(), f"map differs at step {step} {where}"
    for name in ("x", "y"):
        err = np.abs(cur[name][live] - ref_st[name][live])
        assert err.max(initial=0.0) <= TOL_POSE, f"{name} err {err.max()} at step {step} {where}"
    nt = np.nonzero(near)[0]
    if not len(nt):
        return
    sub = np.ascontiguousarray(pre[nt])
    outs = []
    for v in TIE_VARIANTS:
        st = sub.copy()
        o = oracle.step_biased(ocfg, idx[nt], st, actions[nt], *v, nthreads=NTHREADS)
        outs.append((o, st))
    for j, e in enumerate(nt):
        stats.tie(key + (int(idx[e]),), int(pre["episode"][e]), step, step_gap)
        match = [(o["rewards"][j] == rewards[e] and o["dones"][j] == dones[e] and
                  _same_state(cur[e], st[j], bool(o["dones"][j]), S, K)) for o, st in outs]
        assert any(match), f"env {idx[e]} near-tie step {step} {where}: GPU outcome is none of the tie's outcomes"
        exact = (ref["rewards"][e] == rewards[e] and ref["dones"][e] == dones[e] and
                 _same_state(cur[e], ref_st[e], bool(ref["dones"][e]), S, K))
        stats.near_ties_other_way += int(not exact)


def lockstep(run: Run, stats: Stats, n_steps: int, seed: int, first_step: int = 0, idx=None, check_every: int = 1,
             action_fn=inputs.actions):
    """Step the GPU batch; on checked steps, step the oracle from the GPU's
    pre-step state (of envs ``idx``) and compare rewards, dones, poses and
    regenerated episodes; then render the GPU's post-step state in the oracle
    and compare frames and rays."""
    N = run.cfg["n_envs"]
    idx = np.arange(N) if idx is None else np.asarray(idx)
    for s in range(first_step, first_step + n_steps):
        a = action_fn(seed, s, N)
        check = (s - first_step) % check_every == 0
        if check:
            prev = run.state(idx)
        frames, rewards, dones = run.step(a)
        if run.gray is not None:
            run.gray.update(frames, run.env.fields(run.env.get_state())["t"])
        if not check:
            continue
        if run.gray is not None:
            run.gray.check(run.env)
        cur = run.state(idx)
        check_step(run.ocfg, idx, prev, a[idx], cur, rewards[idx], dones[idx], run.env.S, run.env.K, stats, s,
                   step_gap=check_every)
        # render parity on the exact post-step state of the GPU
        rr = render_ref(run.ocfg, cur)
        compare_frames(frames[idx], rr, stats)
        hits, perp = run.rays()
        compare_rays(hits[idx], perp[idx], rr, stats)


def place_facing(f, e, cell, target, on_axis_frac):
    """Put env e's agent in `cell`, facing the adjacent cell `target`."""
    dx, dy = target[0] - cell[0], target[1] - cell[1]
    f["cell_x"][e], f["cell_y"][e] = cell
    f["frac_x"][e] = 0.5 if dx == 0 else (on_axis_frac if dx > 0 else 1.0 - on_axis_frac)
    f["frac_y"][e] = 0.5 if dy == 0 else (on_axis_frac if dy > 0 else 1.0 - on_axis_frac)
    f["theta0"][e] = np.float32(np.arctan2(dy, dx) % (2 * np.pi))
    f["turn"][e] = 0


def script_goal_and_door(f: dict, n: int, S: int):
    """In the state fields f of n maze envs: even envs stand next to their goal
    (key held) facing it, odd envs in front of their door (key held or not)
    facing it. Returns (number of goal walkers, {odd env: door will open})."""
    n_goal, opens = 0, {}
    for e in range(n):
        m = f["map"][e]
        gx, gy, dxc, dyc = (int(v) for v in f["obj"][e][2:6])
        if e % 2 == 0:
            target = (gx, gy)
            f["flags"][e] = 1
            n_goal += 1
        else:
            target = (dxc, dyc)
            f["flags"][e] = (e // 2) % 2
        for ox, oy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            nb = (target[0] + ox, target[1] + oy)
            if 0 <= nb[0] < S and 0 <= nb[1] < S and (m[nb[1], nb[0]] == 0 or
                                                      (m[nb[1], nb[0]] == oracle.DOOR and f["flags"][e])):
                break
        place_facing(f, e, nb, target, 0.45)
        if e % 2:
            key = (int(f["obj"][e][0]), int(f["obj"][e][1]))
            opens[e] = bool(f["flags"][e]) or nb == key  # standing on the key picks it up at once
    return n_goal, opens


def check_door_crossings(before: dict, after: dict, opens: dict):
    """A door walker moved at least one cell iff its door was open to it."""
    for e, will_open in opens.items():
        dist = abs(int(after["cell_x"][e]) - int(before["cell_x"][e])) + abs(
            int(after["cell_y"][e]) - int(before["cell_y"][e]))
        assert (dist >= 1) == will_open, e


class BatchRun:
    """A jx.Batch over fresh envs of the given group configs, with flat torch buffers."""

    def __init__(self, cfgs: list, tiling=None, device: int = 0):
        self.cfgs = cfgs
        self.envs = [jx.Env(c, device) for c in cfgs]
        self.ocfgs = [oracle_cfg(c) for c in cfgs]
        self.batch = jx.Batch(self.envs, tiling)
        dev = torch.device("cuda", device)
        self.dev = dev
        self.frames = torch.zeros(self.batch.frame_bytes, dtype=torch.uint8, device=dev)
        self.rewards = torch.zeros(self.batch.n, dtype=torch.float32, device=dev)
        self.dones = torch.zeros(self.batch.n, dtype=torch.uint8, device=dev)
        self.actions = torch.zeros(self.batch.n, dtype=torch.uint8, device=dev)

    def group_frames(self, frames: np.ndarray, i: int) -> np.ndarray:
        """Group i's [n, H, W, 3] frames out of a flat frame array of one step."""
        env = self.envs[i]
        _, fs = self.batch.group_slices(i)
        return frames[fs].reshape(env.n, env.H, env.W, 3)

    def reset(self):
        self.batch.reset(self.frames)
        torch.cuda.synchronize()
        return self.frames.cpu().numpy()

    def step(self, actions: np.ndarray):
        self.actions.copy_(torch.from_numpy(actions))
        self.batch.step(self.actions, self.frames, self.rewards, self.dones)
        torch.cuda.synchronize()
        return self.frames.cpu().numpy(), self.rewards.cpu().numpy(), self.dones.cpu().numpy()

    def states(self) -> list:
        return [to_oracle(e, e.get_state()) for e in self.envs]


def batch_check_reset(run: BatchRun, stats: Stats):
    frames = run.reset()
    for i, env in enumerate(run.envs):
        gpu = to_oracle(env, env.get_state())
        ref = oracle.generate(run.ocfgs[i], np.arange(env.n, dtype=np.int32), 0, nthreads=NTHREADS)
        compare_generated(gpu, ref, env.S, env.K, f"at batch reset, group {i}")
        compare_frames(run.group_frames(frames, i), render_ref(run.ocfgs[i], gpu), stats)


def batch_lockstep(run: BatchRun, stats: Stats, n_steps: int, seed: int, first_step: int = 0, check_every: int = 1,
                   action_fn=inputs.actions):
    """lockstep() for every group of a batch stepped in one launch per step."""
    N = run.batch.n
    for s in range(first_step, first_step + n_steps):
        a = action_fn(seed, s, N)
        check = (s - first_step) % check_every == 0
        if check:
            prev = run.states()
        frames, rewards, dones = run.step(a)
        if not check:
            continue
        cur = run.states()
        for i, env in enumerate(run.envs):
            es, _ = run.batch.group_slices(i)
            idx = np.arange(env.n, dtype=np.int32)
            check_step(run.ocfgs[i], idx, prev[i], a[es], cur[i], rewards[es], dones[es], env.S, env.K, stats, s,
                       f"group {i}", key=(i,), step_gap=check_every)
            rr = render_ref(run.ocfgs[i], cur[i])
            compare_frames(run.group_frames(frames, i), rr, stats)
