"""The allocation-free host-buffer step, jx_step_host_static.

Some callers cannot allocate device memory when they step: a process whose
device memory a framework's caching allocator already holds, or a loop that
may not take the implicit synchronisation of a first-use cudaMalloc. For them
jx_step_host_static stages through a fixed array inside the library instead
of the buffers jx_step_host allocates on first use. These tests check, through
the C ABI, that it returns exactly what jx_step_host returns on two calls in a
row (the second call ends every episode and regenerates the maps, and runs on
the array the first call left behind) while the device's free memory stays
the same across each call, and that batches too large for the array are
refused. This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_2605_19926_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jx():
    from paper_2605_19926_gb300 import build

    build.build()
    from paper_2605_19926_gb300 import jx as mod

    assert torch.cuda.is_available()
    return mod


def _host_buffers(cfg):
    N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    return (torch.zeros((N, H, W, 3), dtype=torch.uint8).pin_memory(),
            torch.zeros(N, dtype=torch.float32).pin_memory(),
            torch.zeros(N, dtype=torch.uint8).pin_memory())


def test_static_staging_matches_host_step_two_calls(jx):
    cfg = inputs.maze_keydoor(n_envs=300, map_side=32, seed=17, horizon=2)
    N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    ref, new = jx.Env(cfg), jx.Env(cfg)
    dev_frames = torch.zeros((N, H, W, 3), dtype=torch.uint8, device="cuda")
    ref.reset(dev_frames)
    new.reset(dev_frames)
    torch.cuda.synchronize()
    fr, rr, dr = _host_buffers(cfg)
    fn, rn, dn = _host_buffers(cfg)
    for s in range(2):
        act = torch.from_numpy(inputs.actions(23, s, N)).pin_memory()
        ref.step_host(act, fr, rr, dr)  # also loads the step kernel the static call launches
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        new.step_host_static(act, fn, rn, dn)
        torch.cuda.synchronize()
        # the array was reserved when the env was created: the call takes no device memory
        assert torch.cuda.mem_get_info()[0] == free0, f"free device memory changed on call {s}"
        assert torch.equal(fr, fn), f"frames differ on call {s}"
        assert torch.equal(rr, rn) and torch.equal(dr, dn), f"rewards / dones differ on call {s}"
    assert int(dn.sum()) == N  # the second call ended every episode
    assert (ref.get_state() == new.get_state()).all()


def test_static_staging_rejects_oversized_batch(jx):
    cfg = inputs.batched_keydoor_mazes(4096)  # 4096 x 12 KB frames: far beyond the fixed array
    env = jx.Env(cfg)
    N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    act = np.zeros(N, np.uint8)
    frames = np.zeros((N, H, W, 3), np.uint8)
    rewards = np.zeros(N, np.float32)
    dones = np.zeros(N, np.uint8)
    with pytest.raises(jx.JxError) as ei:
        env.step_host_static(act, frames, rewards, dones)
    assert ei.value.status == jx.EINVAL and "staging" in str(ei.value)
