"""Seeded synthetic inputs: workload presets and random action streams.

This module holds no arithmetic of the method. It only names workload
parameters and draws the uniformly random actions that drive an episode
rollout (the paper times its environments under a uniform random policy,
App. A.1). Both the CUDA path and the oracle consume what it produces.
"""

from __future__ import annotations

import numpy as np

N_ACTIONS = 7  # noop, forward, back, strafe-left, strafe-right, turn-left, turn-right

TASK_ROOMS = 0
TASK_MAZE_KEYDOOR = 1
TASK_MAZE_ROOMS = 2
TASK_ASCII = 3

_COMMON = dict(
    frame_h=64,
    frame_w=64,
    turns_per_rev=72,  # 5 degree turns
    fov_deg=60.0,
    move_step=0.1,
    radius=0.2,
)


def rooms(n_envs: int = 1, map_side: int = 16, wall_prob: float = 0.25, seed: int = 0, max_sprites: int = 0,
          frame_h: int = 64, frame_w: int = 64) -> dict:
    """Random-wall rooms: border walls, interior walls with probability ``wall_prob``,
    no reward and no episode end (a single env, 16 x 16 map, 64 x 64 frame by default)."""
    return dict(_COMMON, task=TASK_ROOMS, n_envs=n_envs, map_side=map_side, wall_prob=wall_prob,
                max_sprites=max_sprites, horizon=0, step_reward=0.0, key_reward=0.0, goal_reward=0.0,
                seed=seed, frame_h=frame_h, frame_w=frame_w)


def maze_keydoor(n_envs: int = 4096, map_side: int = 32, seed: int = 1, horizon: int = 500,
                 frame_h: int = 64, frame_w: int = 64) -> dict:
    """Random DFS mazes with one key, one locked door and a goal at the farthest
    cell; +1 key, +10 goal, -0.001 per step, auto-reset after ``horizon`` steps."""
    return dict(_COMMON, task=TASK_MAZE_KEYDOOR, n_envs=n_envs, map_side=map_side, wall_prob=0.0,
                max_sprites=2, horizon=horizon, step_reward=-0.001, key_reward=1.0, goal_reward=10.0,
                seed=seed, frame_h=frame_h, frame_w=frame_w)


# The two workloads the tests and the benchmark run.
def single_env_rooms() -> dict:
    """1 env, 16 x 16 random rooms (p = 0.25), 64 x 64 RGB, 1000 random steps, seed 0."""
    return rooms(n_envs=1, map_side=16, wall_prob=0.25, seed=0)


def batched_keydoor_mazes(n_envs: int = 4096) -> dict:
    """4096 envs, 32 x 32 DFS key-door mazes, 64 x 64 RGB, horizon 500, 10,000 random steps, seed 1."""
    return maze_keydoor(n_envs=n_envs, map_side=32, seed=1, horizon=500)


def maze_rooms(n_envs: int = 65536, map_side: int = 128, seed: int = 4, horizon: int = 500, max_sprites: int = 16,
               frame_h: int = 128, frame_w: int = 128, gray_stack: int = 1) -> dict:
    """Key-door mazes with S*S/1024 open 8 x 8 rooms and up to K - 2 distractor sprites
    (rewards as the key-door maze), RGB frames plus the 4-frame grayscale stack."""
    return dict(maze_keydoor(n_envs=n_envs, map_side=map_side, seed=seed, horizon=horizon, frame_h=frame_h,
                             frame_w=frame_w), task=TASK_MAZE_ROOMS, max_sprites=max_sprites, gray_stack=gray_stack)


def large_scale(n_envs: int = 65536) -> dict:
    """65,536 envs, 128 x 128 mazes with 8 x 8 rooms, 16 sprite slots, 128 x 128 RGB and
    the grayscale stack, horizon 500, 1000-step random-action rollouts, seed 4."""
    return maze_rooms(n_envs=n_envs)


# ASCII maps (Table 2 symbols) of this repository's own design: the paper names
# its ASCII domains (simple, key-door, key-corridor) but prints none of them.
ASCII_MAPS = {
    "simple": "\n".join([
        "############",
        "#S.........#",
        "#..####....#",
        "#.....#....#",
        "#.....#..G.#",
        "############",
    ]),
    "key-door": "\n".join([
        "##########",
        "#S...#...#",
        "#....#.G.#",
        "#.r..R...#",
        "#....#...#",
        "##########",
    ]),
    "coloured-rooms": "\n".join([
        "#################",
        "#S..#...#.....#.#",
        "#...B...\".....Y.#",
        "#.b.#...#..y..#G#",
        "##R###\\#######.#",
        "#...#...#.......#",
        "#.r.#S..1...2..S#",
        "#################",
    ]),
}


def ascii_env(name: str, n_envs: int = 16, map_side: int = 24, seed: int = 6, horizon: int = 200,
              max_sprites: int = 4, frame_h: int = 64, frame_w: int = 64, shading: int = 0) -> dict:
    """An ASCII map of ASCII_MAPS as an env config (+1 per key, +10 at the goal, -0.001 per step)."""
    return dict(_COMMON, task=TASK_ASCII, n_envs=n_envs, map_side=map_side, wall_prob=0.0, max_sprites=max_sprites,
                horizon=horizon, step_reward=-0.001, key_reward=1.0, goal_reward=10.0, seed=seed, frame_h=frame_h,
                frame_w=frame_w, shading=shading, ascii_map=ASCII_MAPS[name])


UNEVEN_SIDES = (16, 32, 64, 128)
UNEVEN_FRAMES = (32, 64, 96, 128)


def uneven_groups(n_envs: int = 16384, seed: int = 2, wall_prob: float = 0.3, max_sprites: int = 8,
                  horizon: int = 0) -> list[dict]:
    """Uneven batch: ``n_envs`` random-wall rooms (p = 0.3), each env's map side drawn
    uniformly from {16, 32, 64, 128} and its square RGB frame size uniformly from
    {32, 64, 96, 128}, 0-8 sprites per env (drawn at each episode start). Envs that
    share (map side, frame size) form one group, i.e. one env config; the groups
    come in (side, frame) order and each has its own seed."""
    rng = np.random.default_rng([int(seed) & 0xFFFFFFFF, 0x4A59])
    side = rng.integers(0, len(UNEVEN_SIDES), size=n_envs)
    frame = rng.integers(0, len(UNEVEN_FRAMES), size=n_envs)
    counts = np.bincount(side * len(UNEVEN_FRAMES) + frame, minlength=len(UNEVEN_SIDES) * len(UNEVEN_FRAMES))
    groups = []
    for k, n in enumerate(counts):
        if n == 0:
            continue
        S, F = UNEVEN_SIDES[k // len(UNEVEN_FRAMES)], UNEVEN_FRAMES[k % len(UNEVEN_FRAMES)]
        g = rooms(n_envs=int(n), map_side=S, wall_prob=wall_prob, seed=int(seed) * 1000 + k, max_sprites=max_sprites,
                  frame_h=F, frame_w=F)
        g["horizon"] = horizon
        groups.append(g)
    return groups


def serving_session(seed: int, actor: int, k: int) -> dict:
    """Session k of actor group `actor` in the serving workload: a batch of envs
    log-uniform in [16, 4096], 32 x 32 or 64 x 64 key-door mazes (even), 64 x 64
    RGB frames, its own seed."""
    rng = np.random.default_rng([int(seed) & 0xFFFFFFFF, int(actor), int(k), 0x4A5A])
    n = int(round(float(np.exp(rng.uniform(np.log(16.0), np.log(4096.0))))))
    side = int(rng.choice([32, 64]))
    return maze_keydoor(n_envs=n, map_side=side, seed=int(seed) * 1_000_003 + actor * 10_007 + k, horizon=500)


def arrival_gaps(seed: int, actor: int, n: int, mean_s: float = 2e-3) -> np.ndarray:
    """Exponential gaps (a Poisson process of mean gap `mean_s`) between one actor group's step requests."""
    rng = np.random.default_rng([int(seed) & 0xFFFFFFFF, int(actor), 0x4A5B])
    return rng.exponential(mean_s, size=n)


def actions(seed: int, step: int, n_envs: int) -> np.ndarray:
    """Uniform random actions in [0, 7) for one step of ``n_envs`` envs (uint8)."""
    rng = np.random.default_rng([int(seed) & 0xFFFFFFFF, int(step) & 0xFFFFFFFF, 0x4A58])
    return rng.integers(0, N_ACTIONS, size=n_envs, dtype=np.uint8)


def action_stream(seed: int, n_steps: int, n_envs: int, first_step: int = 0) -> np.ndarray:
    """[n_steps, n_envs] uint8 actions; row i equals ``actions(seed, first_step + i, n_envs)``."""
    out = np.empty((n_steps, n_envs), np.uint8)
    for i in range(n_steps):
        out[i] = actions(seed, first_step + i, n_envs)
    return out
