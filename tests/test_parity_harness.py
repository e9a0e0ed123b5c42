"""The lockstep parity harness on the CPU: fed the oracle's own results in
place of the GPU's it must pass, and fed a planted mistake (a reward, a pose,
a key, a pixel, a ray's hit) it must fail. Near-tie steps and corner rays are
accepted in either of the ways their tie admits, and in no other way."""
import numpy as np
import pytest

import oracle
from paper_2605_19926_gb300 import inputs
from parity import Stats, check_step, compare_frames, compare_rays, render_ref


def _maze(n=48, seed=7, horizon=9):
    cfg = inputs.maze_keydoor(n_envs=n, map_side=16, seed=seed, horizon=horizon, frame_h=32, frame_w=32)
    return oracle.make_config(**cfg), np.arange(n, dtype=np.int32)


def _walk(ocfg, idx, steps, seed=3):
    """(pre-step states, actions, post-step states, rewards, dones) of an oracle walk."""
    envs = oracle.generate(ocfg, idx)
    out = []
    for s in range(steps):
        a = inputs.actions(seed, s, len(idx))
        pre = envs.copy()
        r = oracle.step(ocfg, idx, envs, a)
        out.append((pre, a, envs.copy(), r["rewards"], r["dones"]))
    return out


def test_oracle_results_pass():
    ocfg, idx = _maze()
    stats = Stats()
    for s, (pre, a, cur, rew, done) in enumerate(_walk(ocfg, idx, 12)):
        check_step(ocfg, idx, pre, a, cur, rew, done, 16, 2, stats, s)
        ref = render_ref(ocfg, cur)
        compare_frames(ref["frames"].copy(), ref, stats)
        rays = ref["rays"]
        hits = np.stack([rays["cell_x"], rays["cell_y"], rays["side"], rays["h"]], axis=-1)
        compare_rays(hits, rays["perp"].astype(np.float32), ref, stats)
    assert stats.resets > 0 and stats.env_steps == 12 * len(idx)
    stats.check()


@pytest.mark.parametrize("plant", ["reward", "done", "x", "keys", "turn", "map"])
def test_planted_step_mistakes_fail(plant):
    ocfg, idx = _maze()
    pre, a, cur, rew, done = _walk(ocfg, idx, 3)[2]
    cur, rew, done = cur.copy(), rew.copy(), done.copy()
    e = 5
    if plant == "reward":
        rew[e] = np.float32(rew[e] + 1.0)
    elif plant == "done":
        done[e] ^= 1
    elif plant == "x":
        cur["x"][e] += 1e-4
    elif plant == "keys":
        cur["keys"][e] ^= 1
    elif plant == "turn":
        cur["turn"][e] = (cur["turn"][e] + 1) % 72
    else:
        cur["map"][e][17] ^= 1
    with pytest.raises(AssertionError):
        check_step(ocfg, idx, pre, a, cur, rew, done, 16, 2, Stats(), 2)


def _tie_case():
    """One env whose forward move ends with the box edge on a wall face."""
    from oracle_helpers import config, empty_room, env_from

    grid = empty_room(8)
    grid[1:-1, 6] = 2
    ocfg = config(S=8)
    return ocfg, env_from(8, grid, 5.7, 3.5, 0.0, 0)


def test_near_tie_step_accepts_either_outcome_only():
    ocfg, pre = _tie_case()
    idx = np.array([0], np.int32)
    a = np.array([1], np.uint8)
    outs = []
    for bias in (1, -1):
        st = pre.copy()
        o = oracle.step_biased(ocfg, idx, st, a, bias, bias, 0, 0)
        assert o["events"][0] & oracle.EV_NEAR_TIE
        outs.append((st, o))
    assert outs[0][0]["x"][0] != outs[1][0]["x"][0]
    stats = Stats()
    for st, o in outs:  # the move and the block both pass
        check_step(ocfg, idx, pre, a, st, o["rewards"], o["dones"], 8, 4, stats, 0)
    assert stats.near_ties == 2
    bad = outs[0][0].copy()
    bad["x"][0] += 0.05  # neither outcome
    with pytest.raises(AssertionError):
        check_step(ocfg, idx, pre, a, bad, outs[0][1]["rewards"], outs[0][1]["dones"], 8, 4, Stats(), 0)


def test_near_tie_runs_count_consecutive_steps_once():
    s = Stats()
    for step in range(5):
        s.tie((0,), 0, step, 1)
    s.tie((0,), 1, 5, 1)  # a new episode: a new run
    s.tie((1,), 0, 5, 1)
    assert s.near_ties == 7 and s.near_tie_runs == 3


def _corner_state():
    import math

    from oracle_helpers import config, empty_room, env_from

    S, W, col = 8, 64, 20
    ocfg = config(S=S, H=64, W=W)
    T = math.tan(math.radians(30.0))
    cx = 2.0 * (col + 0.5) / W - 1.0
    th = math.pi / 4
    rx, ry = math.cos(th) - cx * T * math.sin(th), math.sin(th) + cx * T * math.cos(th)
    grid = empty_room(S)
    grid[2, 3] = 2
    grid[3, 2] = 3
    return ocfg, env_from(S, grid, 3.0 - 0.5 * rx, 3.0 - 0.5 * ry, th, 0), col


@pytest.mark.parametrize("bias", [1, -1])
def test_corner_ray_accepts_either_decision(bias):
    ocfg, st, col = _corner_state()
    ref = render_ref(ocfg, st)
    assert ref["rays"]["corner"][0, col] == 1
    v = oracle.render(ocfg, st, bias=bias)
    frames = ref["frames"].copy()
    frames[0, :, col] = v["frames"][0, :, col]
    r = v["rays"]
    hits = np.stack([r["cell_x"], r["cell_y"], r["side"], r["h"]], axis=-1)
    stats = Stats()
    compare_frames(frames, ref, stats)
    compare_rays(hits, r["perp"].astype(np.float32), ref, stats)
    assert stats.corner_rays >= 1


def test_corner_ray_rejects_a_third_result():
    ocfg, st, col = _corner_state()
    ref = render_ref(ocfg, st)
    r = ref["rays"]
    hits = np.stack([r["cell_x"], r["cell_y"], r["side"], r["h"]], axis=-1)
    hits[0, col, :2] = (4, 4)  # a cell neither decision hits
    with pytest.raises(AssertionError):
        compare_rays(hits, r["perp"].astype(np.float32), ref, Stats())
    frames = ref["frames"].copy()
    frames[0, 10:20, col] = 255  # a column matching neither decision
    with pytest.raises(AssertionError):
        compare_frames(frames, ref, Stats())


def test_planted_pixel_and_ray_mistakes_fail():
    ocfg, idx = _maze(n=8)
    cur = _walk(ocfg, idx, 2)[1][2]
    ref = render_ref(ocfg, cur)
    amb = ref["ambiguous"].astype(bool)
    e, y, x = np.argwhere(~amb)[100]
    frames = ref["frames"].copy()
    frames[e, y, x] ^= 0x40
    with pytest.raises(AssertionError):
        compare_frames(frames, ref, Stats())
    r = ref["rays"]
    ok = np.argwhere(r["corner"] == 0)[3]
    hits = np.stack([r["cell_x"], r["cell_y"], r["side"], r["h"]], axis=-1)
    perp = r["perp"].astype(np.float32)
    hits[tuple(ok)][2] ^= 1
    with pytest.raises(AssertionError):
        compare_rays(hits, perp, ref, Stats())
    hits[tuple(ok)][2] ^= 1
    perp[tuple(ok)] *= 1.001
    with pytest.raises(AssertionError):
        compare_rays(hits, perp, ref, Stats())
