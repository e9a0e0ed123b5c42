"""Pins for the oracle's step: closed-form motion, the collision invariant and
a hand-worked key-door trace."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle_helpers import config, empty_room, env_from

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "keydoor_trace.json")


def _actions(spec):
    out = []
    for part in spec.split(","):
        a, n = part.split("*")
        out += [int(a)] * int(n)
    return out


def _step(orc, cfg, e, a, env_index=0):
    o = orc.step(cfg, np.array([env_index]), e, np.array([a], np.uint8))
    return float(o["rewards"][0]), int(o["dones"][0]), int(o["events"][0])


@pytest.mark.parametrize("trace", json.load(open(GOLDEN))["traces"], ids=lambda t: t["name"])
def test_hand_worked_keydoor_trace(orc, trace):
    g = json.load(open(GOLDEN))
    cfg = orc.make_config(**g["config"])
    # the trace's map notation: '#' wall, '.' floor, '5' the red locked door;
    # its key and goal are the key and goal sprites on those cells
    grid = np.array([[orc.DOOR if ch == "5" else (0 if ch == "." else 1) for ch in row] for row in trace["map"]],
                    np.uint8)
    S = grid.shape[0]
    st = trace["start"]
    sprites = []
    if trace["key"][0] >= 0:
        sprites.append((trace["key"][0] + 0.5, trace["key"][1] + 0.5, orc.SPR_KEY))
    if trace["goal"][0] >= 0:
        sprites.append((trace["goal"][0] + 0.5, trace["goal"][1] + 0.5, orc.SPR_GOAL))
    e = env_from(S, grid, st["x"], st["y"], st["theta0"], st["turn"], sprites=sprites, key=tuple(trace["key"]),
                 goal=tuple(trace["goal"]), door=tuple(trace["door"]))
    ex = trace["expect"]
    keys, goals, dones = [], [], []
    for k, a in enumerate(_actions(trace["actions"]), start=1):
        r, d, ev = _step(orc, cfg, e, a)
        assert not (ev & oracle.EV_NEAR_TIE)
        want_r = ex["reward"].get(str(k), ex["reward"]["default"])
        assert np.float32(r) == np.float32(want_r), k
        if ev & oracle.EV_KEY:
            keys.append(k)
        if ev & oracle.EV_GOAL:
            goals.append(k)
        if d:
            dones.append(k)
            assert e["episode"][0] == 1 and e["t"][0] == 0
            break
        for fld in ("x", "y"):
            want = ex.get(f"{fld}_after", {}).get(str(k))
            if want is not None:
                assert abs(e[fld][0] - want) < 1e-12, (fld, k)
        want = ex.get("turn_after", {}).get(str(k))
        if want is not None:
            assert e["turn"][0] == want
    assert keys == ex["key_steps"] and goals == ex["goal_steps"] and dones == ex["done_steps"]


def test_forward_ten_steps_is_one_cell(orc):
    S = 16
    cfg = config(S=S)
    for turn in (0, 7, 30, 61):
        e = env_from(S, empty_room(S), 7.5, 7.5, 0.3, turn)
        for _ in range(10):
            _step(orc, cfg, e, 1)
        th = 0.3 + turn * 2 * math.pi / 72
        assert abs(e["x"][0] - (7.5 + math.cos(th))) < 1e-12
        assert abs(e["y"][0] - (7.5 + math.sin(th))) < 1e-12


def test_strafe_and_back_directions(orc):
    S = 16
    cfg = config(S=S)
    e = env_from(S, empty_room(S), 7.5, 7.5, 0.0)
    _step(orc, cfg, e, 4)  # strafe right: +y when facing +x (y axis points down)
    assert abs(e["y"][0] - 7.6) < 1e-12 and abs(e["x"][0] - 7.5) < 1e-12
    _step(orc, cfg, e, 3)
    _step(orc, cfg, e, 3)
    assert abs(e["y"][0] - 7.4) < 1e-12
    _step(orc, cfg, e, 2)
    assert abs(e["x"][0] - 7.4) < 1e-12


def test_turns_are_inverse_and_periodic(orc):
    S = 16
    cfg = config(S=S)
    e = env_from(S, empty_room(S), 7.5, 7.5, 1.0, 3)
    for _ in range(72):
        _step(orc, cfg, e, 6)
    assert e["turn"][0] == 3
    for _ in range(5):
        _step(orc, cfg, e, 5)
    assert e["turn"][0] == 70


def _box_overlaps_wall(grid, x, y, r, keys):
    """Open-box overlap with any solid cell (the invariant: never inside a wall)."""
    S = grid.shape[0]
    for j in range(S):
        for i in range(S):
            v = grid[j, i]
            if v == 0 or (v == 16 and keys & 1):
                continue
            if x + r > i and x - r < i + 1 and y + r > j and y - r < j + 1:
                return True
    return False


@pytest.mark.parametrize("task,S", [(0, 16), (1, 16)])
def test_agent_never_inside_a_wall(orc, task, S):
    p = dict(task=task, map_side=S, frame_h=32, frame_w=32, max_sprites=2, horizon=0, turns_per_rev=72,
             fov_deg=60.0, move_step=0.1, radius=0.2, wall_prob=0.35, step_reward=0.0, key_reward=0.0,
             goal_reward=0.0, seed=11)
    cfg = orc.make_config(**p)
    n = 6
    envs = orc.generate(cfg, np.arange(n))
    rng = np.random.default_rng(3)
    moved = 0
    for s in range(400):
        before = envs[["x", "y"]].copy()
        # bias towards forward so the agents reach walls
        acts = np.where(rng.random(n) < 0.6, 1, rng.integers(0, 7, n)).astype(np.uint8)
        orc.step(cfg, np.arange(n), envs, acts)
        moved += int((before["x"] != envs["x"]).sum())
        if s % 10 == 0:
            for i in range(n):
                grid = orc.map_view(cfg, envs[i])
                assert not _box_overlaps_wall(grid, envs["x"][i], envs["y"][i], 0.2, envs["keys"][i])
    assert moved > 100


def test_horizon_and_auto_reset(orc):
    p = dict(task=1, map_side=16, frame_h=32, frame_w=32, max_sprites=2, horizon=7, turns_per_rev=72,
             fov_deg=60.0, move_step=0.1, radius=0.2, wall_prob=0.0, step_reward=-0.001, key_reward=1.0,
             goal_reward=10.0, seed=2)
    cfg = orc.make_config(**p)
    envs = orc.generate(cfg, np.arange(3))
    for s in range(1, 15):
        o = orc.step(cfg, np.arange(3), envs, np.zeros(3, np.uint8))
        assert (o["dones"] == (1 if s % 7 == 0 else 0)).all()
        assert (envs["t"] == s % 7).all()
    assert (envs["episode"] == 2).all()
    fresh = orc.generate(cfg, np.arange(3), 2)
    assert (fresh["map"] == envs["map"]).all()
    assert (fresh["x"] == envs["x"]).all() and (fresh["theta0"] == envs["theta0"]).all()
