"""FP64 CPU oracle of the batched first-person environment step + render.

TEST INFRASTRUCTURE ONLY. This package is the slow, plainly-written statement
of what the GPU path computes (JAXenstein, arxiv 2605.19926: DDA ray casting
over a tile map, Sec. 2.1; wall slices from the hit distance, Sec. 2; fixed
sprites, Fig. 1; keys, locked doors and a goal, Tables 1-2; native
low-resolution frames, Sec. 3.1). Only the test suite, the smoke check and the
benchmark's CPU-baseline / reference leg may import it. It shares no code with
the CUDA library and imports nothing from it.

Parity status of each function is pinned in ``tests/test_oracle_*.py``:
SplitMix64 against published output vectors; the raycaster against closed
forms, mirror symmetry and brute-force fine-step marching; the step against
closed-form motion, the collision invariant and a hand-worked key-door trace;
the generators against spanning-tree / BFS / reachability invariants.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(HERE, "jx_oracle.c")
_LIB_PATH = os.path.join(HERE, "liboracle.so")

MAX_SIDE = 128
MAX_SPRITES = 16

TASK_ROOMS = 0
TASK_MAZE_KEYDOOR = 1
TASK_MAZE_ROOMS = 2
TASK_ASCII = 3

FLOOR = 0
LOCKED = 16  # + colour (0 red, 1 blue, 2 yellow)
UNLOCKED = 20  # + colour
DOOR = LOCKED  # the red locked door of the generated key-door mazes
SPR_KEY, SPR_GOAL, SPR_DISTRACTOR, SPR_KEY_BLUE, SPR_KEY_YELLOW = 1, 2, 3, 4, 5

EV_KEY = 1
EV_GOAL = 2
EV_NEAR_TIE = 4

CONFIG_DTYPE = np.dtype(
    [
        ("task", np.int32),
        ("map_side", np.int32),
        ("frame_h", np.int32),
        ("frame_w", np.int32),
        ("max_sprites", np.int32),
        ("horizon", np.int32),
        ("turns_per_rev", np.int32),
        ("shading", np.int32),
        ("wall_prob", np.float64),
        ("fov_deg", np.float64),
        ("move_step", np.float64),
        ("radius", np.float64),
        ("step_reward", np.float64),
        ("key_reward", np.float64),
        ("goal_reward", np.float64),
        ("seed", np.uint64),
        ("ascii", np.uint64),
    ],
    align=True,
)

ENV_DTYPE = np.dtype(
    [
        ("x", np.float64),
        ("y", np.float64),
        ("theta0", np.float64),
        ("turn", np.int32),
        ("t", np.int32),
        ("episode", np.uint32),
        ("keys", np.int32),
        ("key_x", np.int32),
        ("key_y", np.int32),
        ("goal_x", np.int32),
        ("goal_y", np.int32),
        ("door_x", np.int32),
        ("door_y", np.int32),
        ("n_sprites", np.int32),
        ("pad0", np.int32),
        ("spr_x", np.float64, (MAX_SPRITES,)),
        ("spr_y", np.float64, (MAX_SPRITES,)),
        ("spr_type", np.int32, (MAX_SPRITES,)),
        ("map", np.uint8, (MAX_SIDE * MAX_SIDE,)),
    ],
    align=True,
)

RAY_DTYPE = np.dtype(
    [
        ("cell_x", np.int32),
        ("cell_y", np.int32),
        ("side", np.int32),
        ("h", np.int32),
        ("top", np.int32),
        ("bot", np.int32),
        ("corner", np.int32),
        ("h_ambiguous", np.int32),
        ("perp", np.float64),
    ],
    align=True,
)

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/liboracle.so``."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(HERE, "jx_oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i32, u32, u64 = ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
        L.jxo_splitmix64.argtypes = [u64, u64]
        L.jxo_splitmix64.restype = u64
        L.jxo_draw.argtypes = [u64, u32, u32, u32, u32]
        L.jxo_draw.restype = u64
        for f in ("jxo_sizeof_env", "jxo_sizeof_config", "jxo_sizeof_ray"):
            getattr(L, f).restype = ctypes.c_int
        L.jxo_generate.argtypes = [P, i32, u32, P]
        L.jxo_step.argtypes = [P, i32, P, i32, P, P, P]
        L.jxo_cast.argtypes = [P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, i32, P]
        L.jxo_render.argtypes = [P, P, P, P, P]
        L.jxo_step_render_batch.argtypes = [P, P, P, i32, P, P, P, P, P, P, P, i32]
        L.jxo_render_batch.argtypes = [P, P, i32, P, P, P, i32]
        L.jxo_generate_batch.argtypes = [P, P, P, P, i32, i32]
        L.jxo_render_batch_biased.argtypes = [P, P, i32, P, P, P, i32, i32]
        L.jxo_step_batch_biased.argtypes = [P, P, P, i32, P, i32, i32, i32, i32, P, P, P, i32]
        L.jxo_step_biased.argtypes = [P, i32, P, i32, i32, i32, i32, i32, P, P, P]
        L.jxo_gray.argtypes = [P, ctypes.c_int64, P]
        L.jxo_gray.restype = None
        L.jxo_parse_ascii.argtypes = [ctypes.c_char_p, i32, P]
        L.jxo_sizeof_ascii.restype = ctypes.c_int
        assert L.jxo_sizeof_env() == ENV_DTYPE.itemsize, "oracle env layout mismatch"
        assert L.jxo_sizeof_config() == CONFIG_DTYPE.itemsize, "oracle config layout mismatch"
        assert L.jxo_sizeof_ray() == RAY_DTYPE.itemsize, "oracle ray layout mismatch"
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


_ascii_maps = []  # parsed maps referenced by configs (kept alive for the process)


def parse_ascii(text: str, side: int) -> np.ndarray:
    """The oracle's parse of an ASCII map (Table 2 symbols) laid out in an S x S grid."""
    buf = np.zeros(lib().jxo_sizeof_ascii(), np.uint8)
    if lib().jxo_parse_ascii(text.encode("ascii"), side, _ptr(buf)) != 0:
        raise ValueError("oracle: ASCII map does not parse")
    _ascii_maps.append(buf)
    return buf


def make_config(**params) -> np.ndarray:
    """A one-element CONFIG_DTYPE record; unknown keys (e.g. ``n_envs``) are ignored.
    ``ascii_map`` (text) is parsed by the oracle for the ASCII task."""
    cfg = np.zeros(1, dtype=CONFIG_DTYPE)
    for name in CONFIG_DTYPE.names:
        if name in params and name != "ascii":
            cfg[name] = params[name]
    if params.get("ascii_map") is not None:
        cfg["ascii"] = parse_ascii(params["ascii_map"], int(params["map_side"])).ctypes.data
    return cfg


def splitmix64(seed: int, n: int) -> int:
    return int(lib().jxo_splitmix64(seed & (2**64 - 1), n & (2**64 - 1)))


def draw(seed: int, env: int, episode: int, purpose: int, index: int) -> int:
    return int(lib().jxo_draw(seed & (2**64 - 1), env, episode, purpose, index))


def generate(cfg: np.ndarray, env_index, episode=None, nthreads: int = 1) -> np.ndarray:
    """Episode ``episode`` (default 0) of each env in ``env_index``."""
    env_index = np.ascontiguousarray(np.atleast_1d(env_index), dtype=np.int32)
    n = env_index.size
    episode = np.zeros(n, np.uint32) if episode is None else np.ascontiguousarray(
        np.broadcast_to(np.asarray(episode, np.uint32), (n,)))
    out = np.zeros(n, dtype=ENV_DTYPE)
    rc = lib().jxo_generate_batch(_ptr(cfg), _ptr(env_index), _ptr(episode), _ptr(out), n, nthreads)
    if rc != 0:
        raise ValueError("oracle: invalid config")
    return out


def step(cfg: np.ndarray, env_index, envs: np.ndarray, actions, frames=False, rays=False, ambiguous=False,
         nthreads: int = 1) -> dict:
    """Step every env in ``envs`` in place (auto-reset included) and render.

    Returns rewards (float32, the FP64 reward rounded once), dones (uint8),
    events (int32 bits: 1 key, 2 goal, 4 near-tie) and, if asked, frames
    [n, H, W, 3] uint8, rays [n, W] RAY_DTYPE and ambiguous [n, H, W] uint8.
    """
    env_index = np.ascontiguousarray(np.atleast_1d(env_index), dtype=np.int32)
    n = envs.shape[0]
    actions = np.ascontiguousarray(actions, dtype=np.uint8)
    assert actions.shape == (n,) and env_index.shape == (n,)
    H, W = int(cfg["frame_h"][0]), int(cfg["frame_w"][0])
    out = {
        "rewards": np.zeros(n, np.float32),
        "dones": np.zeros(n, np.uint8),
        "events": np.zeros(n, np.int32),
    }
    if frames:
        out["frames"] = np.zeros((n, H, W, 3), np.uint8)
    if rays:
        out["rays"] = np.zeros((n, W), RAY_DTYPE)
    if ambiguous:
        out["ambiguous"] = np.zeros((n, H, W), np.uint8)
    rc = lib().jxo_step_render_batch(
        _ptr(cfg), _ptr(env_index), _ptr(envs), n, _ptr(actions), _ptr(out["rewards"]), _ptr(out["dones"]),
        _ptr(out["events"]), _ptr(out.get("frames")), _ptr(out.get("rays")), _ptr(out.get("ambiguous")), nthreads)
    if rc != 0:
        raise ValueError("oracle: invalid config or action")
    return out


def render(cfg: np.ndarray, envs: np.ndarray, rays=True, ambiguous=True, nthreads: int = 1, bias: int = 0) -> dict:
    """Frames (and rays, ambiguity flags) of the envs' current states. ``bias``
    +1 / -1 casts every ray with its near ties taken towards the x / y
    boundary: the frame of one of the decisions a corner ray admits."""
    envs = np.ascontiguousarray(envs)
    n = envs.shape[0]
    H, W = int(cfg["frame_h"][0]), int(cfg["frame_w"][0])
    out = {"frames": np.zeros((n, H, W, 3), np.uint8)}
    if rays:
        out["rays"] = np.zeros((n, W), RAY_DTYPE)
    if ambiguous:
        out["ambiguous"] = np.zeros((n, H, W), np.uint8)
    rc = lib().jxo_render_batch_biased(_ptr(cfg), _ptr(envs), n, _ptr(out["frames"]), _ptr(out.get("rays")),
                                       _ptr(out.get("ambiguous")), bias, nthreads)
    if rc != 0:
        raise ValueError("oracle: invalid config or bias")
    return out


def step_biased(cfg: np.ndarray, env_index, envs: np.ndarray, actions, coll_x: int, coll_y: int, pick_x: int,
                pick_y: int, nthreads: int = 1) -> dict:
    """``step`` (no frames) with the decisions a near tie admits taken one way:
    coll_x / coll_y +1 let a collision test within the tie tolerance pass, -1
    block it; pick_x / pick_y shift the key / goal test point by -1, 0 or +1
    times the tolerance. All zero is ``step``."""
    env_index = np.ascontiguousarray(np.atleast_1d(env_index), dtype=np.int32)
    n = envs.shape[0]
    actions = np.ascontiguousarray(actions, dtype=np.uint8)
    assert actions.shape == (n,) and env_index.shape == (n,) and envs.flags["C_CONTIGUOUS"]
    out = {"rewards": np.zeros(n, np.float32), "dones": np.zeros(n, np.uint8), "events": np.zeros(n, np.int32)}
    rc = lib().jxo_step_batch_biased(_ptr(cfg), _ptr(env_index), _ptr(envs), n, _ptr(actions), coll_x, coll_y,
                                     pick_x, pick_y, _ptr(out["rewards"]), _ptr(out["dones"]), _ptr(out["events"]),
                                     nthreads)
    if rc != 0:
        raise ValueError("oracle: invalid config, action or bias")
    return out


def cast(cfg: np.ndarray, env: np.ndarray, ox: float, oy: float, rx: float, ry: float, bias: int = 0) -> np.ndarray:
    """One DDA ray from (ox, oy) along (rx, ry) through ``env``'s map."""
    out = np.zeros(1, RAY_DTYPE)
    e = np.ascontiguousarray(env.reshape(1))
    lib().jxo_cast(_ptr(cfg), _ptr(e), ox, oy, rx, ry, bias, _ptr(out))
    return out[0]


def gray(rgb: np.ndarray) -> np.ndarray:
    """Integer BT.601 luma of an [..., 3] uint8 array: (77 R + 150 G + 29 B + 128) >> 8."""
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
    out = np.empty(rgb.shape[:-1], np.uint8)
    lib().jxo_gray(_ptr(rgb), out.size, _ptr(out))
    return out


def map_view(cfg: np.ndarray, env) -> np.ndarray:
    """The S x S map of one env record as a 2-D array view."""
    S = int(cfg["map_side"][0])
    return env["map"][: S * S].reshape(S, S)
