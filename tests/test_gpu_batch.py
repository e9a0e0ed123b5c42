"""Batched launches over env groups of different sizes (jx_batch_*): the CUDA
path against the FP64 oracle, against each group stepped alone, across
tilings, rollouts, CUDA-graph replay and the autotuner."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_19926_gb300 import inputs, jx
from parity import (NTHREADS, BatchRun, Run, Stats, batch_check_reset, batch_lockstep, check_door_crossings,
                    check_step, compare_frames, compare_generated, forward_biased_actions, render_ref,
                    script_goal_and_door, to_oracle)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_19926_gb300 import build

    build.build()
    assert torch.cuda.is_available()


def mixed():
    """Six groups: every map side and frame size of the uneven workload, the
    room, maze and ASCII tasks, sprites, coloured keys and doors, distance
    shading, episode ends by horizon and by goal."""
    return [
        inputs.rooms(n_envs=7, map_side=16, wall_prob=0.3, seed=21, max_sprites=8, frame_h=32, frame_w=32),
        dict(inputs.rooms(n_envs=3, map_side=128, wall_prob=0.3, seed=22, max_sprites=8, frame_h=128, frame_w=128),
             horizon=25),
        inputs.maze_keydoor(n_envs=9, map_side=32, seed=23, horizon=40),
        inputs.rooms(n_envs=5, map_side=64, wall_prob=0.3, seed=24, max_sprites=8, frame_h=96, frame_w=96),
        inputs.maze_keydoor(n_envs=33, map_side=8, seed=25, horizon=60),
        inputs.ascii_env("coloured-rooms", n_envs=11, map_side=24, seed=26, horizon=70, shading=1, frame_h=48,
                         frame_w=80),
    ]


def tiling(w, c, bits, rows, staging=1):
    t = jx.Tiling()
    t.warps_per_block, t.cols_per_lane, t.bits_min_side, t.max_rows_per_block, t.staging_buffers = (w, c, bits, rows,
                                                                                                   staging)
    return t


TILINGS = {
    "default": None,
    "bits_everywhere_2w_2c_4rows": tiling(2, 2, 8, 4),
    "bytes_everywhere_4w_8rows_2buffers": tiling(4, 1, 0, 8, 2),
}


@pytest.mark.parametrize("name", list(TILINGS))
def test_batch_lockstep_vs_oracle(name):
    run = BatchRun(mixed(), TILINGS[name])
    stats = Stats()
    batch_check_reset(run, stats)
    batch_lockstep(run, stats, 240, seed=31, action_fn=forward_biased_actions)
    stats.check()
    assert stats.key_events > 0 and stats.resets > 0, stats


@pytest.mark.parametrize("name", ["default", "bits_everywhere_2w_2c_4rows"])
def test_batch_scripted_goal_reach_and_door_crossing(name):
    """Maze groups of side 16 and 128 (byte map and bit plane under the default
    tiling; bit planes for both under the other): agents placed next to their
    goal or in front of their door walk forward, in lockstep with the oracle."""
    cfgs = [inputs.maze_keydoor(n_envs=32, map_side=16, seed=13, horizon=0),
            inputs.maze_keydoor(n_envs=8, map_side=128, seed=14, horizon=0, frame_h=96, frame_w=96)]
    run = BatchRun(cfgs, TILINGS[name])
    run.reset()
    before, expect = [], []
    for env in run.envs:
        blob = env.get_state()
        f = env.fields(blob)
        expect.append(script_goal_and_door(f, env.n, env.S))
        env.set_state(blob)
        before.append(f)
    stats = Stats()
    batch_lockstep(run, stats, 20, seed=0, action_fn=lambda seed, step, n: np.ones(n, np.uint8))
    stats.check()
    n_goal = sum(e[0] for e in expect)
    assert stats.goal_events == n_goal and stats.resets == n_goal, stats
    for env, f, (_, opens) in zip(run.envs, before, expect):
        check_door_crossings(f, env.fields(env.get_state()), opens)


def test_batch_equals_groups_alone():
    """Each group's frames, rewards, dones and state are the same stepped alone
    (jx_step of that env) and in the mix (one batched launch)."""
    cfgs = mixed()
    run = BatchRun(cfgs, tiling(2, 2, 32, 8, 2))
    alone = [Run(c) for c in cfgs]
    frames = run.reset()
    for i, a in enumerate(alone):
        a.reset()
        assert (run.group_frames(frames, i) == a.frames.cpu().numpy()).all(), i
    for s in range(70):
        act = forward_biased_actions(41, s, run.batch.n)
        frames, rewards, dones = run.step(act)
        for i, a in enumerate(alone):
            es, _ = run.batch.group_slices(i)
            fa, ra, da = a.step(act[es])
            assert (run.group_frames(frames, i) == fa).all(), (s, i)
            assert (rewards[es] == ra).all() and (dones[es] == da).all(), (s, i)
    for env, a in zip(run.envs, alone):
        assert (env.get_state() == a.env.get_state()).all()
        env.sync_status()  # no bulk map copy (side-64 byte maps) timed out


def _rollout(run: BatchRun, acts: torch.Tensor):
    T = acts.shape[0]
    frames = torch.zeros((T, run.batch.frame_bytes), dtype=torch.uint8, device=run.dev)
    rewards = torch.zeros((T, run.batch.n), dtype=torch.float32, device=run.dev)
    dones = torch.zeros((T, run.batch.n), dtype=torch.uint8, device=run.dev)
    run.batch.rollout(acts, frames, rewards, dones)
    torch.cuda.synchronize()
    return frames, rewards, dones


@pytest.mark.parametrize("name", list(TILINGS))
def test_batch_rollout_matches_step_sequence(name):
    """A rollout launch under any tiling equals T batched steps under the default tiling."""
    cfgs = mixed()
    ref = BatchRun(cfgs)
    run = BatchRun(cfgs, TILINGS[name])
    ref.reset()
    run.reset()
    T = 50
    acts = torch.from_numpy(np.stack([forward_biased_actions(43, s, run.batch.n) for s in range(T)])).to(run.dev)
    frames, rewards, dones = _rollout(run, acts)
    for t in range(T):
        ref.actions.copy_(acts[t])
        ref.batch.step(ref.actions, ref.frames, ref.rewards, ref.dones)
        assert torch.equal(ref.frames, frames[t]), t
        assert torch.equal(ref.rewards, rewards[t]) and torch.equal(ref.dones, dones[t]), t
    torch.cuda.synchronize()
    for a, b in zip(ref.envs, run.envs):
        assert (a.get_state() == b.get_state()).all()
        a.sync_status()
        b.sync_status()
    assert int(dones.sum().item()) > 0


def test_graph_replay_matches_steps():
    cfgs = mixed()
    ref = BatchRun(cfgs)
    run = BatchRun(cfgs, tiling(1, 2, 64, 16))
    ref.reset()
    run.reset()
    T = 12
    acts = torch.from_numpy(np.stack([inputs.actions(47, s, run.batch.n) for s in range(T)])).to(run.dev)
    frames = torch.zeros((T, run.batch.frame_bytes), dtype=torch.uint8, device=run.dev)
    rewards = torch.zeros((T, run.batch.n), dtype=torch.float32, device=run.dev)
    dones = torch.zeros((T, run.batch.n), dtype=torch.uint8, device=run.dev)
    graph = run.batch.capture(acts, frames, rewards, dones)
    n0 = run.batch.launch_count()
    graph.launch()
    torch.cuda.synchronize()
    assert run.batch.launch_count() == n0 + T
    for t in range(T):
        ref.actions.copy_(acts[t])
        ref.batch.step(ref.actions, ref.frames, ref.rewards, ref.dones)
        assert torch.equal(ref.frames, frames[t]), t
        assert torch.equal(ref.rewards, rewards[t]) and torch.equal(ref.dones, dones[t]), t
    torch.cuda.synchronize()
    for a, b in zip(ref.envs, run.envs):
        assert (a.get_state() == b.get_state()).all()
    graph.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_autotune_keeps_fastest_and_resets(mode):
    cfgs = mixed()
    run = BatchRun(cfgs)
    fresh = BatchRun(cfgs)
    fresh.reset()
    run.reset()
    run.step(inputs.actions(3, 0, run.batch.n))
    trials = run.batch.autotune(mode=mode, steps=3, max_trials=9)
    assert len(trials) == 9
    assert trials[0][0].as_tuple() == jx.default_tiling().as_tuple()
    assert all(ms > 0 for _, ms in trials)
    best = min(trials, key=lambda x: x[1])[0]
    assert run.batch.tiling.as_tuple() == best.as_tuple()
    for a, b in zip(fresh.envs, run.envs):  # every env back at its episode-0 start
        assert (a.get_state() == b.get_state()).all()


def test_tiling_validation():
    run = BatchRun(mixed()[:1])
    for bad in (tiling(3, 1, 0, 8), tiling(1, 3, 0, 8), tiling(1, 1, -1, 8), tiling(1, 1, 0, 0), tiling(1, 1, 0, 65),
                tiling(1, 1, 0, 8, 3), tiling(1, 1, 0, 8, 0)):
        with pytest.raises(jx.JxError) as ei:
            run.batch.tiling = bad
        assert ei.value.status == jx.EINVAL
    with pytest.raises(jx.JxError):
        jx.Batch([run.envs[0], run.envs[0]])


def test_full_size_uneven_batch_sampled():
    """16,384 envs of the uneven workload (16 groups: map sides 16..128, frames
    32..128 square, 0-8 sprites) in one launch per step under the autotuned
    tiling: 4 sampled envs of every group checked against the oracle at reset
    and after each of 3 steps, and the rollout of those steps equal to them."""
    cfgs = inputs.uneven_groups()
    run = BatchRun(cfgs)
    run.batch.autotune(mode=1, steps=2, max_trials=12)
    rng = np.random.default_rng(9)
    idx = [np.sort(rng.choice(e.n, min(4, e.n), replace=False)).astype(np.int32) for e in run.envs]
    stats = Stats()
    frames = run.reset()
    for i, env in enumerate(run.envs):
        gpu = to_oracle(env, env.get_state(), idx[i])
        ref = oracle.generate(run.ocfgs[i], idx[i], 0, nthreads=NTHREADS)
        compare_generated(gpu, ref, env.S, env.K, f"group {i}")
        compare_frames(run.group_frames(frames, i)[idx[i]], render_ref(run.ocfgs[i], gpu), stats)
    T = 3
    acts = np.stack([inputs.actions(5, s, run.batch.n) for s in range(T)])
    step_frames = []
    for s in range(T):
        prev = [to_oracle(e, e.get_state(), idx[i]) for i, e in enumerate(run.envs)]
        frames, rewards, dones = run.step(acts[s])
        step_frames.append(frames)
        for i, env in enumerate(run.envs):
            es, _ = run.batch.group_slices(i)
            cur = to_oracle(env, env.get_state(), idx[i])
            check_step(run.ocfgs[i], idx[i], prev[i], acts[s][es][idx[i]], cur, rewards[es][idx[i]],
                       dones[es][idx[i]], env.S, env.K, stats, s, f"group {i}", key=(i,))
            rr = render_ref(run.ocfgs[i], cur)
            compare_frames(run.group_frames(frames, i)[idx[i]], rr, stats)
    stats.check()
    # the same three steps as one rollout launch from a fresh reset
    run.reset()
    rf, _, _ = _rollout(run, torch.from_numpy(acts).to(run.dev))
    for s in range(T):
        assert (rf[s].cpu().numpy() == step_frames[s]).all(), s


@pytest.mark.parametrize("cfg", [inputs.maze_keydoor(n_envs=40, map_side=32, seed=101, horizon=30),
                                 inputs.maze_rooms(n_envs=9, map_side=64, seed=102, horizon=20, frame_h=96,
                                                   frame_w=96)])
def test_env_autotune_and_pinned_tilings_give_identical_results(cfg):
    """jx_autotune times the env's own kernel (trial 0) against batched tilings and
    resets every env; whichever kernel an env is pinned to, its frames, rewards,
    dones and state (grayscale stack included) are the same."""
    ref, tuned = Run(cfg), Run(cfg)
    trials = tuned.env.autotune(mode=1, steps=3, max_trials=6)
    assert len(trials) == 6 and trials[0][0].as_tuple() == (0, 0, 0, 0, 0)
    best = min(trials, key=lambda x: x[1])[0].as_tuple()
    assert tuned.env.tiling.as_tuple() == best
    ref.reset()
    assert (ref.env.get_state() == tuned.env.get_state()).all()
    pins = [tiling(4, 2, 8, 4), None, tiling(1, 1, 0, 16, 2)]
    tuned.reset()
    for s in range(36):
        if s % 12 == 0:
            tuned.env.tiling = pins[s // 12]
        act = forward_biased_actions(103, s, cfg["n_envs"])
        fa, ra, da = ref.step(act)
        fb, rb, db = tuned.step(act)
        assert (fa == fb).all() and (ra == rb).all() and (da == db).all(), s
    assert (ref.env.get_state() == tuned.env.get_state()).all()
