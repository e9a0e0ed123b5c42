"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point the header declares, and validates configurations before
touching CUDA."""
import ctypes
import os
import re
import subprocess

import pytest
import torch

from paper_2605_19926_gb300 import build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "jx.h")


@pytest.fixture(scope="module")
def jx():
    build.build()
    from paper_2605_19926_gb300 import jx as mod

    return mod


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:jx_status|const char\*)\s+(jx_\w+)\s*\(", text, re.M)))


def test_header_declares_expected_entry_points(jx):
    assert _declared() == sorted(jx.SYMBOLS)


def test_library_exports_every_declared_symbol(jx):
    out = subprocess.run(["nm", "-D", "--defined-only", jx.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (jx_\w+)$", out, re.M))
    for name in _declared():
        assert name in exported, name
        assert getattr(jx.lib, name) is not None


def test_field_enum_matches_header(jx):
    text = open(HEADER).read()
    enum = dict((m.group(1).lower(), int(m.group(2))) for m in re.finditer(r"JX_F_(\w+) = (\d+)", text))
    assert enum.pop("count") == len(jx.FIELDS)
    assert {k: v[0] for k, v in jx.FIELDS.items()} == enum


def test_config_struct_matches_header(jx):
    text = open(HEADER).read()
    body = re.search(r"typedef struct \{(.*?)\} jx_config;", text, re.S).group(1)
    names = []
    for decl in re.findall(r"^\s*(?:int32_t|double|uint64_t)\s+([^;]+);", body, re.M):
        names += [n.strip() for n in decl.split(",")]
    assert names == [f[0] for f in jx.Config._fields_]
    assert ctypes.sizeof(jx.Config) == 8 * 4 + 7 * 8 + 8 + 8  # gray_stack and shading


BAD = [
    (dict(n_envs=0), "n_envs"),
    (dict(task=7), "task"),
    (dict(map_side=2), "map_side"),
    (dict(map_side=129), "map_side"),
    (dict(frame_w=40), "frame_w"),
    (dict(frame_w=272), "frame_w"),
    (dict(frame_h=0), "frame_h"),
    (dict(max_sprites=17), "max_sprites"),
    (dict(turns_per_rev=0), "turns_per_rev"),
    (dict(fov_deg=180.0), "fov_deg"),
    (dict(move_step=0.6), "move_step"),
    (dict(radius=0.5), "radius"),
    (dict(wall_prob=1.5), "wall_prob"),
    (dict(horizon=-1), "horizon"),
    (dict(step_reward=float("nan")), "rewards"),
]


@pytest.mark.parametrize("patch,word", BAD)
def test_invalid_config_rejected_before_cuda(jx, patch, word):
    cfg = dict(inputs.rooms(n_envs=4), **patch)
    st, msg = jx.validate_config(cfg)
    assert st == jx.EINVAL and word in msg


def test_maze_constraints(jx):
    for patch in (dict(map_side=7), dict(map_side=4), dict(max_sprites=1)):
        st, msg = jx.validate_config(dict(inputs.maze_keydoor(n_envs=4), **patch))
        assert st == jx.EINVAL, patch


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU failure path")
def test_valid_config_without_gpu_fails_loudly(jx):
    st, msg = jx.validate_config(inputs.batched_keydoor_mazes(16))
    assert st == jx.ECUDA and msg
    with pytest.raises(jx.JxError):
        jx.Env(inputs.single_env_rooms())


def test_tiling_struct_and_default(jx):
    text = open(HEADER).read()
    body = re.search(r"typedef struct \{([^}]*)\} jx_tiling;", text).group(1)
    names = re.findall(r"^\s*int32_t\s+(\w+);", body, re.M)
    assert names == [f[0] for f in jx.Tiling._fields_]
    assert jx.default_tiling().as_tuple() == (1, 1, 128, 32, 1)


def test_batch_arguments_checked_before_cuda(jx):
    h = ctypes.c_void_p()
    assert jx.lib.jx_batch_create(None, 1, None, ctypes.byref(h)) == jx.EINVAL
    arr = (ctypes.c_void_p * 1)(None)
    assert jx.lib.jx_batch_create(arr, 1, None, ctypes.byref(h)) == jx.EINVAL
    assert jx.lib.jx_batch_create(arr, 0, None, ctypes.byref(h)) == jx.EINVAL
    assert jx.lib.jx_batch_create(arr, 33, None, ctypes.byref(h)) == jx.EINVAL
    assert jx.lib.jx_batch_step(None, None, None, None, None, None) == jx.EINVAL
    assert jx.lib.jx_graph_launch(None, None) == jx.EINVAL
    assert jx.lib.jx_batch_destroy(None) == jx.OK and jx.lib.jx_graph_destroy(None) == jx.OK


def test_uneven_workload_groups():
    groups = inputs.uneven_groups()
    assert sum(g["n_envs"] for g in groups) == 16384
    assert len(groups) == 16
    assert {(g["map_side"], g["frame_w"]) for g in groups} == {(s, f) for s in inputs.UNEVEN_SIDES
                                                               for f in inputs.UNEVEN_FRAMES}
    for g in groups:
        assert g["frame_h"] == g["frame_w"] and g["task"] == inputs.TASK_ROOMS
        assert g["wall_prob"] == 0.3 and g["max_sprites"] == 8
        assert 800 < g["n_envs"] < 1250  # 1024 expected per (side, frame) pair
    assert len({g["seed"] for g in groups}) == 16
    assert inputs.uneven_groups() == groups  # seeded


def test_server_arguments_checked_before_cuda(jx):
    h = ctypes.c_void_p()
    assert jx.lib.jx_server_create(0, 0, 4, 2, 64, None, ctypes.byref(h)) == jx.EINVAL  # budget
    assert jx.lib.jx_server_create(0, 1 << 20, 0, 2, 64, None, ctypes.byref(h)) == jx.EINVAL  # sessions
    assert jx.lib.jx_server_create(0, 1 << 20, 4, 0, 64, None, ctypes.byref(h)) == jx.EINVAL  # in flight
    assert jx.lib.jx_server_create(0, 1 << 20, 4, 17, 64, None, ctypes.byref(h)) == jx.EINVAL
    assert jx.lib.jx_server_create(0, 1 << 20, 4, 2, 129, None, ctypes.byref(h)) == jx.EINVAL  # map side
    assert jx.lib.jx_server_submit(None, 1, None, None) == jx.EINVAL
    assert jx.lib.jx_server_wait(None, 0, 0.0) == jx.EINVAL
    assert jx.lib.jx_server_destroy(None) == jx.OK


def test_server_counters_struct_matches_header(jx):
    text = open(HEADER).read()
    body = re.search(r"typedef struct \{([^}]*)\} jx_server_counters;", text).group(1)
    names = re.findall(r"^\s*(?:u?int\d+_t)\s+(\w+);", body, re.M)
    assert names == [f[0] for f in jx.ServerCounters._fields_]


def test_serving_inputs():
    """Serving sessions: batch sizes log-uniform in [16, 4096], map sides 32 or 64,
    64 x 64 key-door mazes; Poisson arrivals with a 2 ms mean gap; all seeded."""
    import numpy as np

    sessions = [inputs.serving_session(3, a, k) for a in range(64) for k in range(8)]
    n = np.array([s["n_envs"] for s in sessions])
    assert n.min() >= 16 and n.max() <= 4096
    logs = np.log(n)
    assert abs(logs.mean() - (np.log(16) + np.log(4096)) / 2) < 0.3
    assert {s["map_side"] for s in sessions} == {32, 64}
    assert all(s["frame_h"] == s["frame_w"] == 64 and s["task"] == inputs.TASK_MAZE_KEYDOOR for s in sessions)
    assert len({s["seed"] for s in sessions}) == len(sessions)
    assert inputs.serving_session(3, 5, 2) == sessions[5 * 8 + 2]
    gaps = inputs.arrival_gaps(3, 7, 20000)
    assert abs(gaps.mean() - 2e-3) < 1e-4 and (gaps > 0).all()
    assert (inputs.arrival_gaps(3, 7, 20000) == gaps).all()
