"""The continuous-batching step server (jx_server_*): results are the same
alone and in the mix, admission follows the byte budget, launches overlap,
waits are bounded, and the frames match the oracle."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2605_19926_gb300 import inputs, jx
from parity import NTHREADS, Run, Stats, compare_frames, render_ref, to_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_19926_gb300 import build

    build.build()
    assert torch.cuda.is_available()


def configs():
    return [
        inputs.maze_keydoor(n_envs=16, map_side=32, seed=51, horizon=30),
        inputs.maze_keydoor(n_envs=300, map_side=64, seed=52, horizon=40),
        dict(inputs.rooms(n_envs=1000, map_side=32, wall_prob=0.3, seed=53, max_sprites=8), horizon=25),
        inputs.maze_keydoor(n_envs=4096, map_side=32, seed=54, horizon=500),
        inputs.ascii_env("key-door", n_envs=40, map_side=16, seed=55, horizon=60, shading=1),
    ]


def _copy(sess):
    torch.cuda.synchronize()
    return sess.frames.clone(), sess.rewards.clone(), sess.dones.clone()


def test_results_same_alone_and_in_the_mix():
    """Sessions of different sizes stepped through the server, their requests
    held back and released together so that they share launches, give the
    frames, rewards and dones of each config stepped alone with jx_step."""
    cfgs = configs()
    with jx.Server(budget_bytes=1 << 30, max_inflight=3) as server:
        sessions = [server.open(c) for c in cfgs]
        alone = [Run(c) for c in cfgs]
        for sess, a in zip(sessions, alone):
            a.reset()
            assert torch.equal(_copy(sess)[0], a.frames)
        for r in range(40):
            acts = [inputs.actions(61 + i, r, s.n) for i, s in enumerate(sessions)]
            mixed = r % 2 == 0
            if mixed:
                server.pause(True)
            tickets = [s.submit(a) for s, a in zip(sessions, acts)]
            if mixed:
                server.pause(False)
            for t in tickets:
                server.wait(t, timeout=30.0)
            for sess, a, act in zip(sessions, alone, acts):
                f, rw, d = _copy(sess)
                fa, ra, da = a.step(act)
                assert (f.cpu().numpy() == fa).all(), r
                assert (rw.cpu().numpy() == ra).all() and (d.cpu().numpy() == da).all(), r
        for sess, a in zip(sessions, alone):
            assert (sess.env.get_state() == a.env.get_state()).all()
        st = server.stats()
        assert st["requests_done"] == 40 * len(cfgs)
        assert st["groups_launched"] > st["launches"]  # requests did share launches
        for sess in sessions:
            sess.close()


def test_admission_follows_the_budget():
    cfg = inputs.maze_keydoor(n_envs=512, map_side=64, seed=71, horizon=500)
    one = None
    with jx.Server(budget_bytes=1 << 30, max_sessions=8) as probe:
        s = probe.open(cfg)
        one = probe.stats()["bytes_in_use"]
        s.close()
    assert 512 * (64 * 64 + 64 * 64 * 3) < one < 1 << 30
    with jx.Server(budget_bytes=2 * one + one // 2, max_sessions=8) as server:
        a, b = server.open(cfg), server.open(cfg)
        assert server.try_open(cfg) is None
        st = server.stats()
        assert st["rejected_opens"] == 1 and st["sessions_open"] == 2 and st["bytes_in_use"] == 2 * one
        t = a.submit(np.ones(512, np.uint8))
        a.close()  # frees once its request has run
        server.wait(t, timeout=30.0)
        c = server.open(cfg)
        assert server.stats()["sessions_open"] == 2
        for s in (b, c):
            s.close()
        assert server.stats()["bytes_in_use"] == 0
    with jx.Server(budget_bytes=1 << 30, max_sessions=1) as server:
        s = server.open(cfg)
        with pytest.raises(jx.JxError) as ei:
            server.open(cfg)
        assert ei.value.status == jx.EBUDGET
        s.close()


def test_launches_overlap_and_stay_exact():
    """A long launch (16,384 envs, 128 x 128 frames) is on the device when a
    second session's request arrives: the second goes out on another launch
    slot at once, and both sessions' results match each env stepped alone."""
    big = inputs.rooms(n_envs=16384, map_side=64, wall_prob=0.3, seed=81, max_sprites=8, frame_h=128, frame_w=128)
    small = inputs.maze_keydoor(n_envs=64, map_side=32, seed=82, horizon=50)
    with jx.Server(budget_bytes=4 << 30, max_inflight=4) as server:
        sb, ss = server.open(big), server.open(small)
        rb, rs = Run(big), Run(small)
        rb.reset()
        rs.reset()
        for r in range(6):
            ab, as_ = inputs.actions(83, r, big["n_envs"]), inputs.actions(84, r, small["n_envs"])
            n0 = server.stats()["launches"]
            tb = sb.submit(ab)
            t0 = time.perf_counter()
            while server.stats()["launches"] == n0 and time.perf_counter() - t0 < 5.0:
                pass  # the big request is on the device
            ts = ss.submit(as_)
            server.wait(tb, timeout=30.0)
            server.wait(ts, timeout=30.0)
            torch.cuda.synchronize()
            for sess, run, act in ((sb, rb, ab), (ss, rs, as_)):
                run.actions.copy_(torch.from_numpy(act))
                run.env.step(run.actions, run.frames, run.rewards, run.dones)
                torch.cuda.synchronize()
                assert torch.equal(sess.frames, run.frames), r
                assert torch.equal(sess.rewards, run.rewards) and torch.equal(sess.dones, run.dones), r
        assert server.stats()["peak_inflight_launches"] >= 2
        sb.close()
        ss.close()


def test_wait_is_bounded():
    cfg = inputs.maze_keydoor(n_envs=8, map_side=32, seed=91, horizon=500)
    with jx.Server(budget_bytes=1 << 28) as server:
        s = server.open(cfg)
        server.pause(True)
        t = s.submit(np.zeros(8, np.uint8))
        with pytest.raises(jx.JxError) as ei:
            server.wait(t, timeout=0.05)
        assert ei.value.status == jx.ETIMEOUT
        server.pause(False)
        server.wait(t, timeout=30.0)
        s.close()


def test_served_frames_match_oracle():
    cfg = inputs.maze_keydoor(n_envs=24, map_side=64, seed=95, horizon=20)
    ocfg = oracle.make_config(**cfg)
    stats = Stats()
    with jx.Server(budget_bytes=1 << 28) as server:
        s = server.open(cfg)
        for r in range(30):
            server.wait(s.submit(inputs.actions(96, r, 24)), timeout=30.0)
            torch.cuda.synchronize()
            ref = render_ref(ocfg, to_oracle(s.env, s.env.get_state()))
            compare_frames(s.frames.cpu().numpy(), ref, stats)
        s.close()
    stats.check()
