"""Helpers that build hand-made environments for the oracle pin tests."""
import numpy as np

import oracle

COMMON = dict(frame_h=64, frame_w=64, turns_per_rev=72, fov_deg=60.0, move_step=0.1, radius=0.2,
              step_reward=-0.001, key_reward=1.0, goal_reward=10.0, seed=5)


def config(task=0, S=16, H=64, W=64, max_sprites=4, horizon=0, **kw):
    p = dict(COMMON, task=task, map_side=S, frame_h=H, frame_w=W, max_sprites=max_sprites, horizon=horizon)
    p.update(kw)
    return oracle.make_config(**p)


def empty_room(S=16, wall=1):
    m = np.zeros((S, S), np.uint8)
    m[0, :] = m[-1, :] = m[:, 0] = m[:, -1] = wall
    return m


def env_from(S, grid, x, y, theta0=0.0, turn=0, sprites=(), key=(-1, -1), goal=(-1, -1), door=(-1, -1),
             keys=0):
    e = np.zeros(1, oracle.ENV_DTYPE)
    e["x"], e["y"], e["theta0"], e["turn"] = x, y, theta0, turn
    flat = np.zeros(oracle.MAX_SIDE * oracle.MAX_SIDE, np.uint8)
    flat[: S * S] = np.asarray(grid, np.uint8).reshape(-1)
    e["map"][0] = flat
    e["key_x"], e["key_y"] = key
    e["goal_x"], e["goal_y"] = goal
    e["door_x"], e["door_y"] = door
    e["keys"] = keys
    e["n_sprites"] = len(sprites)
    for i, (sx, sy, st) in enumerate(sprites):
        e["spr_x"][0, i], e["spr_y"][0, i], e["spr_type"][0, i] = sx, sy, st
    return e
