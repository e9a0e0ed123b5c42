"""Thin ctypes binding over ``libjx.so`` (the C ABI in ``include/jx.h``).

Argument marshalling only: every step of the environment runs in the CUDA
kernels behind the C ABI. Tensors are passed as raw device pointers, streams
as ``cudaStream_t`` handles. There is no CPU fallback: importing this module
raises when the compiled library is missing, and every compute call raises
``JxError`` when the library reports a failure (for example, no GPU).
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjx.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUDGET, EDEVICE = range(7)
TASK_ROOMS, TASK_MAZE_KEYDOOR, TASK_MAZE_ROOMS, TASK_ASCII = 0, 1, 2, 3
LOCKED, UNLOCKED = 16, 20

# State fields (JX_F_*), name -> (index, numpy dtype, per-env shape builder)
FIELDS = {
    "cell_x": (0, np.int16), "cell_y": (1, np.int16), "frac_x": (2, np.float32), "frac_y": (3, np.float32),
    "theta0": (4, np.float32), "turn": (5, np.int16), "t": (6, np.int32), "episode": (7, np.uint32),
    "flags": (8, np.uint8), "obj": (9, np.int16), "nspr": (10, np.uint8), "spr_x": (11, np.float32),
    "spr_y": (12, np.float32), "spr_type": (13, np.uint8), "map": (14, np.uint8), "cos0": (15, np.float32),
    "sin0": (16, np.float32), "gray": (17, np.uint8),
}

# Entry points declared in include/jx.h (checked by the ABI test).
SYMBOLS = [
    "jx_create", "jx_create_ascii", "jx_destroy", "jx_reset", "jx_step", "jx_rollout", "jx_render", "jx_step_host",
    "jx_step_host_static", "jx_debug_rays", "jx_debug_wait_limit", "jx_debug_handoff_limit",
    "jx_state_bytes", "jx_state_field", "jx_get_state", "jx_set_state", "jx_sync_status", "jx_launch_count",
    "jx_rollout_shape",
    "jx_launch_shape", "jx_last_error",
    "jx_tiling_default", "jx_batch_create", "jx_batch_destroy", "jx_batch_info", "jx_batch_group",
    "jx_batch_set_tiling", "jx_batch_get_tiling", "jx_batch_launch_shape", "jx_batch_launch_count",
    "jx_batch_reset", "jx_batch_step", "jx_batch_rollout", "jx_batch_render", "jx_batch_autotune",
    "jx_batch_capture", "jx_graph_launch", "jx_graph_destroy",
    "jx_env_bytes", "jx_create_in", "jx_autotune", "jx_env_tiling", "jx_env_set_tiling",
    "jx_server_create", "jx_server_destroy", "jx_server_open", "jx_server_open_ascii", "jx_server_close",
    "jx_server_session",
    "jx_server_submit", "jx_server_wait", "jx_server_pause", "jx_server_stats", "jx_server_latencies",
]


class JxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"jx status {status}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [
        ("n_envs", ctypes.c_int32), ("task", ctypes.c_int32), ("map_side", ctypes.c_int32),
        ("frame_h", ctypes.c_int32), ("frame_w", ctypes.c_int32), ("max_sprites", ctypes.c_int32),
        ("horizon", ctypes.c_int32), ("turns_per_rev", ctypes.c_int32), ("wall_prob", ctypes.c_double),
        ("fov_deg", ctypes.c_double), ("move_step", ctypes.c_double), ("radius", ctypes.c_double),
        ("step_reward", ctypes.c_double), ("key_reward", ctypes.c_double), ("goal_reward", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("gray_stack", ctypes.c_int32), ("shading", ctypes.c_int32),
    ]

    @classmethod
    def from_dict(cls, d: dict) -> "Config":
        c = cls()
        for name, _ in cls._fields_:
            if name in d:
                setattr(c, name, d[name])
        return c


class Tiling(ctypes.Structure):
    """Tile choices of the batched kernel (``jx_tiling``)."""

    _fields_ = [("warps_per_block", ctypes.c_int32), ("cols_per_lane", ctypes.c_int32),
                ("bits_min_side", ctypes.c_int32), ("max_rows_per_block", ctypes.c_int32),
                ("staging_buffers", ctypes.c_int32)]

    def as_tuple(self) -> tuple[int, int, int, int, int]:
        return (self.warps_per_block, self.cols_per_lane, self.bits_min_side, self.max_rows_per_block,
                self.staging_buffers)

    def __repr__(self):
        return ("Tiling(warps_per_block=%d, cols_per_lane=%d, bits_min_side=%d, max_rows_per_block=%d, "
                "staging_buffers=%d)" % self.as_tuple())


class ServerCounters(ctypes.Structure):
    """Counters of a step server (``jx_server_counters``)."""

    _fields_ = [("requests_submitted", ctypes.c_uint64), ("requests_done", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("env_steps", ctypes.c_uint64), ("groups_launched", ctypes.c_uint64),
                ("rejected_opens", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64),
                ("bytes_in_use", ctypes.c_uint64), ("peak_bytes_in_use", ctypes.c_uint64),
                ("sessions_open", ctypes.c_int32), ("peak_sessions", ctypes.c_int32),
                ("inflight_launches", ctypes.c_int32), ("peak_inflight_launches", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2605_19926_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
    sig = {
        "jx_create": [P, ctypes.c_int, P],
        "jx_create_ascii": [P, ctypes.c_char_p, ctypes.c_int, P],
        "jx_destroy": [P],
        "jx_reset": [P, P, P],
        "jx_step": [P, P, P, P, P, P],
        "jx_rollout": [P, P, P, i32, P, P, P],
        "jx_render": [P, P, P],
        "jx_step_host": [P, P, P, P, P, P],
        "jx_step_host_static": [P, P, P, P, P, P],
        "jx_debug_rays": [P, P, P, P],
        "jx_debug_wait_limit": [P, i32],
        "jx_debug_handoff_limit": [P, i32],
        "jx_state_bytes": [P, P],
        "jx_state_field": [P, i32, P, P],
        "jx_get_state": [P, P, sz],
        "jx_set_state": [P, P, sz],
        "jx_sync_status": [P, P],
        "jx_launch_count": [P, P],
        "jx_launch_shape": [P, P, P, P],
        "jx_rollout_shape": [P, i32, P, P, P, P],
        "jx_tiling_default": [P],
        "jx_batch_create": [P, i32, P, P],
        "jx_batch_destroy": [P],
        "jx_batch_info": [P, P, P],
        "jx_batch_group": [P, i32, P, P],
        "jx_batch_set_tiling": [P, P],
        "jx_batch_get_tiling": [P, P],
        "jx_batch_launch_shape": [P, P, P, P],
        "jx_batch_launch_count": [P, P],
        "jx_batch_reset": [P, P, P],
        "jx_batch_step": [P, P, P, P, P, P],
        "jx_batch_rollout": [P, P, P, i32, P, P, P],
        "jx_batch_render": [P, P, P],
        "jx_batch_autotune": [P, P, i32, i32, i32, P, P, P],
        "jx_batch_capture": [P, i32, P, P, P, P, P],
        "jx_graph_launch": [P, P],
        "jx_graph_destroy": [P],
        "jx_env_bytes": [P, ctypes.c_int, P],
        "jx_autotune": [P, P, i32, i32, i32, P, P, P],
        "jx_env_tiling": [P, P],
        "jx_env_set_tiling": [P, P],
        "jx_create_in": [P, ctypes.c_int, P, sz, P],
        "jx_server_create": [ctypes.c_int, ctypes.c_uint64, i32, i32, i32, P, P],
        "jx_server_destroy": [P],
        "jx_server_open": [P, P, P],
        "jx_server_open_ascii": [P, P, ctypes.c_char_p, P],
        "jx_server_close": [P, i32],
        "jx_server_session": [P, i32, P, P, P, P],
        "jx_server_submit": [P, i32, P, P],
        "jx_server_wait": [P, ctypes.c_uint64, ctypes.c_double],
        "jx_server_pause": [P, i32],
        "jx_server_stats": [P, P],
        "jx_server_latencies": [P, P, ctypes.c_uint64, P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.jx_last_error.argtypes = []
    L.jx_last_error.restype = ctypes.c_char_p
    return L


lib = _load()


def last_error() -> str:
    return lib.jx_last_error().decode()


def _check(status: int):
    if status != OK:
        raise JxError(status, last_error())


def _ptr(t) -> int | None:
    """Raw pointer of a torch tensor / numpy array / int."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


@dataclass
class Shape:
    grid: int
    block: int
    smem: int


class Env:
    """N environments on one GPU (``jx_create`` ... ``jx_destroy``)."""

    def __init__(self, cfg: dict, device: int = 0):
        """``cfg["ascii_map"]`` (text) is the map of the ASCII task."""
        self.cfg = dict(cfg)
        self._c = Config.from_dict(cfg)
        h = ctypes.c_void_p()
        if cfg.get("ascii_map") is not None:
            _check(lib.jx_create_ascii(ctypes.byref(self._c), cfg["ascii_map"].encode("ascii"), device,
                                       ctypes.byref(h)))
        else:
            _check(lib.jx_create(ctypes.byref(self._c), device, ctypes.byref(h)))
        self._h = h
        self.device = device
        self.n = int(cfg["n_envs"])
        self.H, self.W, self.S, self.K = int(cfg["frame_h"]), int(cfg["frame_w"]), int(cfg["map_side"]), int(
            cfg["max_sprites"])

    @classmethod
    def view(cls, handle: int, cfg: dict, device: int = 0) -> "Env":
        """An Env over a handle owned elsewhere (a server session): state access
        and launches, never destroyed by this object."""
        self = cls.__new__(cls)
        self.cfg = dict(cfg)
        self._c = Config.from_dict(cfg)
        self._h = ctypes.c_void_p(handle)
        self._owned = False
        self.device = device
        self.n = int(cfg["n_envs"])
        self.H, self.W, self.S, self.K = int(cfg["frame_h"]), int(cfg["frame_w"]), int(cfg["map_side"]), int(
            cfg["max_sprites"])
        return self

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value and getattr(self, "_owned", True):
            lib.jx_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------- compute
    def reset(self, frames, stream=None):
        _check(lib.jx_reset(self._h, _stream(stream), _ptr(frames)))

    def step(self, actions, frames, rewards, dones, stream=None):
        _check(lib.jx_step(self._h, _stream(stream), _ptr(actions), _ptr(frames), _ptr(rewards), _ptr(dones)))

    def rollout(self, actions, frames, rewards, dones, stream=None):
        """``actions.shape[0]`` steps in one launch (outputs shaped [steps, N, ...])."""
        steps = int(actions.shape[0])
        _check(lib.jx_rollout(self._h, _stream(stream), _ptr(actions), steps, _ptr(frames), _ptr(rewards),
                              _ptr(dones)))

    def render(self, frames, stream=None):
        _check(lib.jx_render(self._h, _stream(stream), _ptr(frames)))

    def step_host(self, actions, frames, rewards, dones, stream=None):
        _check(lib.jx_step_host(self._h, _stream(stream), _ptr(actions), _ptr(frames), _ptr(rewards), _ptr(dones)))

    def step_host_static(self, actions, frames, rewards, dones, stream=None):
        """``step_host`` staging through the library's fixed device array (no allocation)."""
        _check(lib.jx_step_host_static(self._h, _stream(stream), _ptr(actions), _ptr(frames), _ptr(rewards),
                                       _ptr(dones)))

    def debug_rays(self, hits, perp, stream=None):
        _check(lib.jx_debug_rays(self._h, _stream(stream), _ptr(hits), _ptr(perp)))

    def debug_wait_limit(self, rounds: int):
        """Polls before a bulk map copy counts as late (0: every copy is late)."""
        _check(lib.jx_debug_wait_limit(self._h, int(rounds)))

    def debug_handoff_limit(self, polls: int):
        """Polls before a rollout hand-off wait counts as late (0: every wait is late)."""
        _check(lib.jx_debug_handoff_limit(self._h, int(polls)))

    def sync_status(self, stream=None):
        _check(lib.jx_sync_status(self._h, _stream(stream)))

    # ------------------------------------------------------------------ state
    def state_bytes(self) -> int:
        n = ctypes.c_size_t()
        _check(lib.jx_state_bytes(self._h, ctypes.byref(n)))
        return n.value

    def field(self, name: str) -> tuple[int, int]:
        off, nb = ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib.jx_state_field(self._h, FIELDS[name][0], ctypes.byref(off), ctypes.byref(nb)))
        return off.value, nb.value

    def get_state(self) -> np.ndarray:
        buf = np.empty(self.state_bytes(), np.uint8)
        _check(lib.jx_get_state(self._h, buf.ctypes.data, buf.nbytes))
        return buf

    def set_state(self, buf: np.ndarray):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib.jx_set_state(self._h, buf.ctypes.data, buf.nbytes))

    def fields(self, blob: np.ndarray) -> dict:
        """Views of every state field inside a ``get_state`` blob."""
        out = {}
        N, K, S = self.n, self.K, self.S
        shapes = {"obj": (N, 6), "spr_x": (N, K), "spr_y": (N, K), "spr_type": (N, K), "map": (N, S, S),
                  "gray": (N, 4, self.H, self.W) if self.cfg.get("gray_stack") else (0,)}
        for name, (_, dt) in FIELDS.items():
            off, nb = self.field(name)
            a = blob[off: off + nb].view(dt)
            out[name] = a.reshape(shapes.get(name, (N,)))
        return out

    # ------------------------------------------------------------------- info
    def launch_count(self) -> int:
        n = ctypes.c_uint64()
        _check(lib.jx_launch_count(self._h, ctypes.byref(n)))
        return n.value

    def launch_shape(self) -> Shape:
        g, b, s = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib.jx_launch_shape(self._h, ctypes.byref(g), ctypes.byref(b), ctypes.byref(s)))
        return Shape(g.value, b.value, s.value)

    def rollout_shape(self, steps: int) -> tuple[Shape, int]:
        """Launch shape of a jx_rollout of `steps` steps and its steps per hand-off chunk."""
        g, b, s, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib.jx_rollout_shape(self._h, steps, ctypes.byref(g), ctypes.byref(b), ctypes.byref(s),
                                    ctypes.byref(c)))
        return Shape(g.value, b.value, s.value), c.value

    def autotune(self, mode: int = 1, steps: int = 8, max_trials: int = 1000, stream=None):
        """Time the env's own kernel (trial 0) against the batched kernel's tilings; keep
        the fastest; every env is reset. Returns [(Tiling, ms_per_step)]."""
        trials = (Tiling * max_trials)()
        ms = (ctypes.c_float * max_trials)()
        n = ctypes.c_int32()
        _check(lib.jx_autotune(self._h, _stream(stream), mode, steps, max_trials, ctypes.byref(n), trials, ms))
        return [(trials[i], float(ms[i])) for i in range(n.value)]

    @property
    def tiling(self) -> "Tiling":
        """All zero while the env's own kernel runs, else the batched kernel's tiling."""
        t = Tiling()
        _check(lib.jx_env_tiling(self._h, ctypes.byref(t)))
        return t

    @tiling.setter
    def tiling(self, t: "Tiling | None"):
        _check(lib.jx_env_set_tiling(self._h, ctypes.byref(t if t is not None else Tiling())))


def default_tiling() -> Tiling:
    t = Tiling()
    _check(lib.jx_tiling_default(ctypes.byref(t)))
    return t


class Graph:
    """A captured sequence of batched steps (``jx_batch_capture``)."""

    def __init__(self, handle: ctypes.c_void_p, batch: "Batch"):
        self._h = handle
        self._batch = batch  # the graph must not outlive its batch

    def launch(self, stream=None):
        _check(lib.jx_graph_launch(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.jx_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Env groups of different sizes stepped in one launch (``jx_batch_*``).

    The groups are ``Env`` objects; the batch keeps references to them. The
    arrays of a batched call hold every group's envs in the order given:
    ``group_slices`` gives each group's env range and frame byte range.
    """

    def __init__(self, groups: list, tiling: Tiling | None = None):
        self.groups = list(groups)
        arr = (ctypes.c_void_p * len(self.groups))(*[g._h.value for g in self.groups])
        h = ctypes.c_void_p()
        _check(lib.jx_batch_create(arr, len(self.groups), ctypes.byref(tiling) if tiling is not None else None,
                                   ctypes.byref(h)))
        self._h = h
        n, f = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.jx_batch_info(self._h, ctypes.byref(n), ctypes.byref(f)))
        self.n, self.frame_bytes = n.value, f.value
        self.env_offsets, self.frame_offsets = [], []
        for i in range(len(self.groups)):
            eo, fo = ctypes.c_int64(), ctypes.c_int64()
            _check(lib.jx_batch_group(self._h, i, ctypes.byref(eo), ctypes.byref(fo)))
            self.env_offsets.append(eo.value)
            self.frame_offsets.append(fo.value)

    def group_slices(self, i: int) -> tuple[slice, slice]:
        g = self.groups[i]
        e0, f0 = self.env_offsets[i], self.frame_offsets[i]
        return slice(e0, e0 + g.n), slice(f0, f0 + g.n * 3 * g.H * g.W)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.jx_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def reset(self, frames, stream=None):
        _check(lib.jx_batch_reset(self._h, _stream(stream), _ptr(frames)))

    def step(self, actions, frames, rewards, dones, stream=None):
        _check(lib.jx_batch_step(self._h, _stream(stream), _ptr(actions), _ptr(frames), _ptr(rewards), _ptr(dones)))

    def rollout(self, actions, frames, rewards, dones, stream=None):
        steps = int(actions.shape[0])
        _check(lib.jx_batch_rollout(self._h, _stream(stream), _ptr(actions), steps, _ptr(frames), _ptr(rewards),
                                    _ptr(dones)))

    def render(self, frames, stream=None):
        _check(lib.jx_batch_render(self._h, _stream(stream), _ptr(frames)))

    @property
    def tiling(self) -> Tiling:
        t = Tiling()
        _check(lib.jx_batch_get_tiling(self._h, ctypes.byref(t)))
        return t

    @tiling.setter
    def tiling(self, t: Tiling):
        _check(lib.jx_batch_set_tiling(self._h, ctypes.byref(t)))

    def autotune(self, mode: int = 0, steps: int = 4, max_trials: int = 1000, stream=None):
        """Time the tilings of the search space; keeps the fastest and resets every env.

        Returns [(Tiling, ms_per_step)] in trial order (the default tiling first).
        """
        cap = max_trials
        trials = (Tiling * cap)()
        ms = (ctypes.c_float * cap)()
        n = ctypes.c_int32()
        _check(lib.jx_batch_autotune(self._h, _stream(stream), mode, steps, max_trials, ctypes.byref(n), trials, ms))
        return [(trials[i], float(ms[i])) for i in range(n.value)]

    def capture(self, actions, frames, rewards, dones) -> Graph:
        steps = int(actions.shape[0])
        h = ctypes.c_void_p()
        _check(lib.jx_batch_capture(self._h, steps, _ptr(actions), _ptr(frames), _ptr(rewards), _ptr(dones),
                                    ctypes.byref(h)))
        return Graph(h, self)

    def launch_shape(self) -> Shape:
        g, b, s = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib.jx_batch_launch_shape(self._h, ctypes.byref(g), ctypes.byref(b), ctypes.byref(s)))
        return Shape(g.value, b.value, s.value)

    def launch_count(self) -> int:
        n = ctypes.c_uint64()
        _check(lib.jx_batch_launch_count(self._h, ctypes.byref(n)))
        return n.value


class _DeviceArray:
    """A view of library-owned device memory for ``torch.as_tensor``."""

    def __init__(self, ptr: int, shape: tuple, typestr: str, device: int):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3,
                                         "strides": None, "stream": None}
        self.device = device


def device_view(ptr: int, shape: tuple, dtype, device: int):
    """torch tensor aliasing `ptr` (no copy); valid while the owner keeps the memory."""
    import torch

    typestr = {np.uint8: "|u1", np.float32: "<f4"}[dtype]
    with torch.cuda.device(device):
        return torch.as_tensor(_DeviceArray(ptr, shape, typestr, device), device=torch.device("cuda", device))


class Session:
    """An open server session: its config and views of its device outputs."""

    def __init__(self, server: "Server", sid: int, cfg: dict):
        self.server, self.id, self.cfg = server, sid, dict(cfg)
        self.n = int(cfg["n_envs"])
        env, fr, rw, dn = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib.jx_server_session(server._h, sid, ctypes.byref(env), ctypes.byref(fr), ctypes.byref(rw),
                                     ctypes.byref(dn)))
        self.env_handle = env.value
        self.env = Env.view(env.value, cfg, server.device)
        H, W = int(cfg["frame_h"]), int(cfg["frame_w"])
        d = server.device
        self.frames = device_view(fr.value, (self.n, H, W, 3), np.uint8, d)
        self.rewards = device_view(rw.value, (self.n,), np.float32, d)
        self.dones = device_view(dn.value, (self.n,), np.uint8, d)

    def submit(self, actions: np.ndarray) -> int:
        a = np.ascontiguousarray(actions, dtype=np.uint8)
        assert a.shape == (self.n,)
        t = ctypes.c_uint64()
        _check(lib.jx_server_submit(self.server._h, self.id, a.ctypes.data, ctypes.byref(t)))
        return t.value

    def close(self):
        _check(lib.jx_server_close(self.server._h, self.id))


class Server:
    """Continuous-batching step server (``jx_server_*``)."""

    def __init__(self, budget_bytes: int, max_sessions: int = 256, max_inflight: int = 4, max_map_side: int = 64,
                 tiling: Tiling | None = None, device: int = 0):
        h = ctypes.c_void_p()
        _check(lib.jx_server_create(device, int(budget_bytes), max_sessions, max_inflight, max_map_side,
                                    ctypes.byref(tiling) if tiling is not None else None, ctypes.byref(h)))
        self._h = h
        self.device = device

    def open(self, cfg: dict) -> Session:
        """Admit a session; raises JxError (status EBUDGET) when it does not fit now."""
        c = Config.from_dict(cfg)
        sid = ctypes.c_int32()
        if cfg.get("ascii_map") is not None:
            _check(lib.jx_server_open_ascii(self._h, ctypes.byref(c), cfg["ascii_map"].encode("ascii"),
                                            ctypes.byref(sid)))
        else:
            _check(lib.jx_server_open(self._h, ctypes.byref(c), ctypes.byref(sid)))
        return Session(self, sid.value, cfg)

    def try_open(self, cfg: dict) -> Session | None:
        try:
            return self.open(cfg)
        except JxError as e:
            if e.status == EBUDGET:
                return None
            raise

    def wait(self, ticket: int, timeout: float = 10.0):
        _check(lib.jx_server_wait(self._h, ticket, timeout))

    def pause(self, paused: bool = True):
        _check(lib.jx_server_pause(self._h, int(paused)))

    def stats(self) -> dict:
        c = ServerCounters()
        _check(lib.jx_server_stats(self._h, ctypes.byref(c)))
        return c.as_dict()

    def latencies(self) -> np.ndarray:
        out, chunk = [], 1 << 16
        buf = np.empty(chunk, np.float64)
        while True:
            n = ctypes.c_uint64()
            _check(lib.jx_server_latencies(self._h, buf.ctypes.data, chunk, ctypes.byref(n)))
            out.append(buf[: n.value].copy())
            if n.value < chunk:
                return np.concatenate(out)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.jx_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def validate_config(cfg: dict) -> tuple[int, str]:
    """Run ``jx_create``'s validation (which precedes any CUDA call) on ``cfg``.

    Returns (status, message); a valid config on a machine without a GPU
    returns ECUDA from the device query that follows validation.
    """
    c = Config.from_dict(cfg)
    h = ctypes.c_void_p()
    st = lib.jx_create(ctypes.byref(c), 0, ctypes.byref(h))
    if st == OK:
        lib.jx_destroy(h)
    return st, last_error()
