"""CUDA path vs the FP64 oracle, through the C ABI, on seeded synthetic inputs."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_19926_gb300 import inputs, jx
from parity import (NTHREADS, Run, Stats, check_door_crossings, check_reset, check_step, compare_frames,
                    compare_generated, compare_rays, forward_biased_actions, lockstep, render_ref, script_goal_and_door,
                    to_oracle)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_19926_gb300 import build

    build.build()
    assert torch.cuda.is_available()


CASES = {
    "rooms16": inputs.rooms(n_envs=5, map_side=16, wall_prob=0.25, seed=0),
    "rooms16_sprites_40x48": inputs.rooms(n_envs=33, map_side=16, wall_prob=0.3, seed=4, max_sprites=8, frame_h=40,
                                          frame_w=48),
    "maze32_ragged": inputs.maze_keydoor(n_envs=37, map_side=32, seed=1, horizon=60),
    "maze8_events": inputs.maze_keydoor(n_envs=64, map_side=8, seed=3, horizon=120),
    "maze6_events": inputs.maze_keydoor(n_envs=64, map_side=6, seed=5, horizon=120),
    "maze18_96x128": inputs.maze_keydoor(n_envs=9, map_side=18, seed=7, horizon=30, frame_h=96, frame_w=128),
    "mazerooms64_gray": inputs.maze_rooms(n_envs=12, map_side=64, seed=8, horizon=25, max_sprites=16, frame_h=64,
                                          frame_w=64),
    "mazerooms128_gray_128x128": inputs.maze_rooms(n_envs=5, map_side=128, seed=9, horizon=20),
    "mazerooms32_gray_48x80": inputs.maze_rooms(n_envs=21, map_side=32, seed=10, horizon=15, max_sprites=6,
                                                frame_h=48, frame_w=80),
    "ascii_simple_shaded": inputs.ascii_env("simple", n_envs=24, map_side=16, shading=1, horizon=80),
    "ascii_keydoor": inputs.ascii_env("key-door", n_envs=40, map_side=16, horizon=120),
    "ascii_coloured_rooms_shaded": inputs.ascii_env("coloured-rooms", n_envs=48, map_side=24, seed=9, horizon=150,
                                                    shading=1, frame_h=48, frame_w=80),
    "maze32_shaded_gray": dict(inputs.maze_keydoor(n_envs=20, map_side=32, seed=11, horizon=40), shading=1,
                               gray_stack=1),
    "ascii_coloured_rooms_128": dict(inputs.ascii_env("coloured-rooms", n_envs=6, map_side=128, seed=3, horizon=60),
                                     gray_stack=1),
}


@pytest.mark.parametrize("name", list(CASES))
def test_reset_matches_oracle(name):
    run = Run(CASES[name])
    stats = Stats()
    check_reset(run, stats)
    stats.check()


def test_single_env_rooms_1000_steps():
    """1 env, 16 x 16 random rooms, 64 x 64, 1000 uniform random steps, seed 0."""
    cfg = inputs.single_env_rooms()
    run = Run(cfg)
    stats = Stats()
    check_reset(run, stats)
    lockstep(run, stats, 1000, seed=0)
    stats.check()


@pytest.mark.parametrize("name,steps", [("maze32_ragged", 150), ("maze8_events", 300), ("maze6_events", 300),
                                        ("rooms16_sprites_40x48", 120), ("maze18_96x128", 70),
                                        ("mazerooms64_gray", 60), ("mazerooms128_gray_128x128", 45),
                                        ("mazerooms32_gray_48x80", 40), ("ascii_simple_shaded", 120),
                                        ("ascii_keydoor", 200), ("ascii_coloured_rooms_shaded", 200),
                                        ("maze32_shaded_gray", 60), ("ascii_coloured_rooms_128", 80)])
def test_lockstep(name, steps):
    run = Run(CASES[name])
    stats = Stats()
    check_reset(run, stats)
    events = name.endswith("_events") or name in ("ascii_keydoor", "ascii_coloured_rooms_shaded")
    walk = events or name.startswith("ascii")
    lockstep(run, stats, steps, seed=11, action_fn=forward_biased_actions if walk else inputs.actions)
    stats.check()
    if events:
        assert stats.key_events > 0 and stats.resets > 0, stats
    if name in ("maze32_ragged", "maze18_96x128", "maze32_shaded_gray") or name.startswith("mazerooms"):
        assert stats.resets > 0


def test_full_size_batched_mazes_sampled():
    """4096 envs, 32 x 32 key-door mazes, 64 x 64 frames, in the benchmark's launch
    shape: 64 sampled envs checked in lockstep around the start and across the
    500-step horizon (all envs reset there)."""
    cfg = inputs.batched_keydoor_mazes()
    run = Run(cfg)
    stats = Stats()
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(cfg["n_envs"], 64, replace=False))
    idx[-1] = cfg["n_envs"] - 1
    check_reset(run, stats, idx)
    lockstep(run, stats, 8, seed=1, first_step=0, idx=idx)
    lockstep(run, stats, 488, seed=1, first_step=8, idx=idx, check_every=61)
    lockstep(run, stats, 8, seed=1, first_step=496, idx=idx)
    assert stats.resets >= 60
    stats.check()


def test_full_size_all_envs_200_steps():
    """All 4096 envs of the benchmark's workload checked against the oracle:
    the reset, then 200 steps with every 25th step stepped and rendered by the
    oracle from the GPU's pre-step state."""
    cfg = inputs.batched_keydoor_mazes()
    run = Run(cfg)
    stats = Stats()
    check_reset(run, stats)
    lockstep(run, stats, 200, seed=1, check_every=25)
    assert stats.env_steps == 8 * cfg["n_envs"]
    stats.check()


def test_full_size_10000_steps_sampled():
    """The benchmark's workload run for 10,000 steps through jx_rollout in its
    launch shape (128 steps per launch); every 1024 steps, 64 sampled envs take
    two steps in lockstep with the oracle (pre-step state from the GPU). Every
    env crosses the 500-step horizon about 20 times."""
    cfg = inputs.batched_keydoor_mazes()
    N, H, W, T = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"], 128
    run = Run(cfg)
    stats = Stats()
    rng = np.random.default_rng(17)
    idx = np.sort(rng.choice(N, 64, replace=False))
    check_reset(run, stats, idx)
    frames = torch.empty((T, N, H, W, 3), dtype=torch.uint8, device=run.dev)
    rewards = torch.empty((T, N), dtype=torch.float32, device=run.dev)
    dones = torch.empty((T, N), dtype=torch.uint8, device=run.dev)
    s, n_done, launches = 0, 0, 0
    while s < 10000:
        acts = torch.from_numpy(inputs.action_stream(1, T, N, first_step=s)).to(run.dev)
        run.env.rollout(acts, frames, rewards, dones)
        n_done += int(dones.sum().item())
        s += T
        launches += 1
        if launches % 8 == 0 or s >= 10000:
            lockstep(run, stats, 2, seed=1, first_step=s, idx=idx)
            s += 2
    del frames
    run.env.sync_status()
    assert stats.env_steps == 2 * 64 * 10
    ep = run.state(np.arange(N))["episode"]
    assert ep.min() >= 19 and n_done >= 19 * N
    stats.check()


def test_render_only_and_state_roundtrip():
    cfg = inputs.maze_keydoor(n_envs=20, map_side=16, seed=2, horizon=0)
    run = Run(cfg)
    run.reset()
    for s in range(30):
        run.step(inputs.actions(9, s, 20))
    blob = run.env.get_state()
    run.env.set_state(blob)
    assert (run.env.get_state() == blob).all()
    run.env.render(run.frames)
    torch.cuda.synchronize()
    gpu = run.frames.cpu().numpy()
    ref = render_ref(run.ocfg, to_oracle(run.env, blob))
    stats = Stats()
    compare_frames(gpu, ref, stats)
    stats.check()


def test_degenerate_poses_axis_rays_and_boundaries():
    """Rays exactly along the axes, positions exactly on cell boundaries, key held."""
    cfg = inputs.maze_keydoor(n_envs=8, map_side=16, seed=6, horizon=0)
    run = Run(cfg)
    run.reset()
    blob = run.env.get_state()
    f = run.env.fields(blob)
    f["theta0"][:] = 0.0
    f["turn"][:] = np.arange(8) * 9  # multiples of 45 degrees
    f["frac_x"][::2] = 0.0
    f["frac_y"][1::2] = 0.0
    f["flags"][4:] = 1
    run.env.set_state(blob)
    run.env.render(run.frames)
    torch.cuda.synchronize()
    ref = render_ref(run.ocfg, to_oracle(run.env, blob))
    stats = Stats()
    compare_frames(run.frames.cpu().numpy(), ref, stats)
    hits, perp = run.rays()
    compare_rays(hits, perp, ref, stats)
    stats.check()


def test_open_border_takes_the_bounds_test():
    """Rays skip the bounds test only while the staged map's border is solid and
    the agent's cell is inside it. Maps with holes in the border (set through
    jx_set_state: floor cells, and a locked door of a held key) and an agent on
    a border cell must still read cells outside the map as wall 1, as the
    oracle does: frames, rays and lockstep steps, in single steps and in a
    rollout long enough for hand-off chunks."""
    cfg = inputs.maze_keydoor(n_envs=8, map_side=16, seed=14, horizon=0)
    S = cfg["map_side"]

    def opened(run):
        run.reset()
        blob = run.env.get_state()
        f = run.env.fields(blob)
        m = f["map"]
        m[0, 0, 1:S - 1] = 0  # top row open
        m[1, 1:S - 1, S - 1] = 0  # right column open
        m[2, 5, 0] = 16  # a red locked door on the border, its key held
        f["flags"][2] = 1
        m[3, 0, 3:8] = 0  # an agent standing on an opened border cell
        m[3, 1, 3:8] = 0
        f["cell_x"][3], f["cell_y"][3], f["frac_x"][3], f["frac_y"][3] = 5, 0, 0.5, 0.5
        f["turn"][:] = np.arange(8) * 9
        f["turn"][3] = 54  # facing -y: every ray leaves through the top
        run.env.set_state(blob)
        return blob

    run = Run(cfg)
    blob = opened(run)
    run.env.render(run.frames)
    torch.cuda.synchronize()
    ref = render_ref(run.ocfg, to_oracle(run.env, blob))
    stats = Stats()
    compare_frames(run.frames.cpu().numpy(), ref, stats)
    hits, perp = run.rays()
    compare_rays(hits, perp, ref, stats)
    assert (hits[3, :, 1] == -1).sum() >= 16  # env 3's central rays left the map at the top
    lockstep(run, stats, 30, seed=5)
    stats.check()
    # the same steps in one rollout launch (hand-off chunks) equal single steps
    a, b = Run(cfg), Run(cfg)
    opened(a)
    opened(b)
    T, N, H, W = 70, cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    acts = torch.from_numpy(inputs.action_stream(15, T, N)).to(b.dev)
    frames = torch.zeros((T, N, H, W, 3), dtype=torch.uint8, device=b.dev)
    rewards = torch.zeros((T, N), dtype=torch.float32, device=b.dev)
    dones = torch.zeros((T, N), dtype=torch.uint8, device=b.dev)
    b.env.rollout(acts, frames, rewards, dones)
    for t in range(T):
        a.actions.copy_(acts[t])
        a.env.step(a.actions, a.frames, a.rewards, a.dones)
        assert torch.equal(a.frames, frames[t]), t
    torch.cuda.synchronize()
    assert (a.env.get_state() == b.env.get_state()).all()
    a.env.sync_status()
    b.env.sync_status()


@pytest.mark.parametrize("patch", [dict(wall_prob=1.0), dict(wall_prob=0.0), dict(horizon=1), dict(move_step=0.0),
                                   dict(radius=0.0)])
def test_edge_configs(patch):
    cfg = dict(inputs.rooms(n_envs=6, map_side=12, seed=8, max_sprites=3), **patch)
    run = Run(cfg)
    stats = Stats()
    check_reset(run, stats)
    lockstep(run, stats, 40, seed=2)
    stats.check()


def test_max_sizes():
    """128 x 128 maze, 16 sprite slots, 256 x 256 frames."""
    cfg = dict(inputs.maze_keydoor(n_envs=3, map_side=128, seed=12, horizon=0, frame_h=256, frame_w=256),
               max_sprites=16)
    run = Run(cfg)
    stats = Stats()
    check_reset(run, stats)
    lockstep(run, stats, 5, seed=3)
    stats.check()


def test_invalid_action_is_reported_and_ignored():
    from paper_2605_19926_gb300 import jx

    cfg = inputs.rooms(n_envs=4, map_side=12, seed=1)
    run = Run(cfg)
    run.reset()
    before = run.env.get_state()
    run.step(np.array([9, 0, 0, 200], np.uint8))
    with pytest.raises(jx.JxError) as ei:
        run.env.sync_status()
    assert ei.value.status == jx.EDEVICE
    run.env.sync_status()  # cleared
    after = run.env.fields(run.env.get_state())
    b = run.env.fields(before)
    assert (after["frac_x"] == b["frac_x"]).all() and (after["t"] == b["t"] + 1).all()


def test_late_bulk_map_copy_is_reported_and_results_unchanged():
    """Byte maps of 4 KB or more reach shared memory by one bulk copy whose
    wait is bounded. With the first wait's limit at 0 every copy counts as
    late: the kernel waits on (bounded) until the copy lands, records bit 2 of
    the error word, and its steps and rollouts equal those of the default
    limit, bit for bit. (A copy that never lands cannot be made on a healthy
    device; its path skips the env and is not run here.)"""
    from paper_2605_19926_gb300 import jx

    cfg = inputs.rooms(n_envs=96, map_side=68, wall_prob=0.3, seed=31, max_sprites=4)  # 68 x 68 byte maps
    a, b = Run(cfg), Run(cfg)
    b.env.debug_wait_limit(0)
    a.reset()
    b.reset()
    for s in range(10):
        act = inputs.actions(31, s, cfg["n_envs"])
        fa, ra, da = a.step(act)
        fb, rb, db = b.step(act)
        assert (fa == fb).all() and (ra == rb).all() and (da == db).all(), s
    T, N = 6, cfg["n_envs"]
    acts = torch.from_numpy(inputs.action_stream(32, T, N)).to(a.dev)
    outs = []
    for run in (a, b):
        fr = torch.zeros((T, N, cfg["frame_h"], cfg["frame_w"], 3), dtype=torch.uint8, device=run.dev)
        rw = torch.zeros((T, N), dtype=torch.float32, device=run.dev)
        dn = torch.zeros((T, N), dtype=torch.uint8, device=run.dev)
        run.env.rollout(acts, fr, rw, dn)
        torch.cuda.synchronize()
        outs.append((fr.cpu(), rw.cpu(), dn.cpu()))
    assert all(torch.equal(x, y) for x, y in zip(*outs))
    assert (a.env.get_state() == b.env.get_state()).all()
    a.env.sync_status()
    with pytest.raises(jx.JxError) as ei:
        b.env.sync_status()
    assert ei.value.status == jx.EDEVICE and "late" in str(ei.value)
    b.env.sync_status()  # cleared
    with pytest.raises(jx.JxError):
        b.env.debug_wait_limit(-1)
    # the batched kernel's late path: a batch over an env with the limit at 0
    # steps like the env kernel, and its work queues stay usable
    c, d = Run(cfg), Run(cfg)
    c.env.debug_wait_limit(0)
    c.reset()
    d.reset()
    t = jx.Tiling()
    (t.warps_per_block, t.cols_per_lane, t.bits_min_side, t.max_rows_per_block, t.staging_buffers) = (2, 1, 0, 16, 1)
    batch = jx.Batch([c.env], t)
    bf = torch.zeros((N, cfg["frame_h"], cfg["frame_w"], 3), dtype=torch.uint8, device=c.dev)
    for s in range(3):
        act = inputs.actions(33, s, N)
        c.actions.copy_(torch.from_numpy(act))
        batch.step(c.actions, bf, c.rewards, c.dones)
        fd, rd, dd = d.step(act)
        torch.cuda.synchronize()
        assert (bf.cpu().numpy() == fd).all() and (c.rewards.cpu().numpy() == rd).all(), s
    with pytest.raises(jx.JxError):
        c.env.sync_status()
    batch.close()


def test_step_host_matches_device_step():
    cfg = inputs.maze_keydoor(n_envs=50, map_side=16, seed=4, horizon=25)
    a, b = Run(cfg), Run(cfg)
    a.reset()
    b.reset()
    hf = torch.zeros((50, 64, 64, 3), dtype=torch.uint8).pin_memory()
    hr = torch.zeros(50, dtype=torch.float32).pin_memory()
    hd = torch.zeros(50, dtype=torch.uint8).pin_memory()
    for s in range(60):
        act = inputs.actions(4, s, 50)
        f, r, d = a.step(act)
        b.env.step_host(torch.from_numpy(act), hf, hr, hd)
        assert (hf.numpy() == f).all() and (hr.numpy() == r).all() and (hd.numpy() == d).all()


def test_same_seed_same_frames():
    cfg = inputs.maze_keydoor(n_envs=16, map_side=16, seed=21, horizon=20)
    a, b = Run(cfg), Run(cfg)
    a.reset()
    b.reset()
    for s in range(45):
        act = inputs.actions(3, s, 16)
        fa, ra, da = a.step(act)
        fb, rb, db = b.step(act)
        assert (fa == fb).all() and (ra == rb).all() and (da == db).all()


def test_scripted_goal_reach_and_door_crossing():
    """Agents placed next to their goal (even envs) or in front of their door
    (odd envs, key held or not) walk forward; checked in lockstep."""
    cfg = inputs.maze_keydoor(n_envs=32, map_side=16, seed=13, horizon=0)
    run = Run(cfg)
    run.reset()
    blob = run.env.get_state()
    f = run.env.fields(blob)
    n_goal, opens = script_goal_and_door(f, 32, 16)
    run.env.set_state(blob)
    stats = Stats()
    lockstep(run, stats, 20, seed=0, action_fn=lambda seed, step, n: np.ones(n, np.uint8))
    stats.check()
    assert stats.goal_events == n_goal and stats.resets == n_goal, stats
    check_door_crossings(f, run.env.fields(run.env.get_state()), opens)


def _rollout_vs_steps(cfg, T, seed, warm=0):
    """jx_rollout over T steps equals T jx_step calls, bit for bit (frames,
    rewards, dones and the final state); both start from the same state."""
    N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    a, b = Run(cfg), Run(cfg)
    a.reset()
    b.reset()
    for s in range(warm):
        act = inputs.actions(seed, s, N)
        a.step(act)
        b.step(act)
    acts = torch.from_numpy(inputs.action_stream(seed, T, N, first_step=warm)).to(a.dev)
    frames = torch.zeros((T, N, H, W, 3), dtype=torch.uint8, device=a.dev)
    rewards = torch.zeros((T, N), dtype=torch.float32, device=a.dev)
    dones = torch.zeros((T, N), dtype=torch.uint8, device=a.dev)
    b.env.rollout(acts, frames, rewards, dones)
    torch.cuda.synchronize()
    for t in range(T):
        a.actions.copy_(acts[t])
        a.env.step(a.actions, a.frames, a.rewards, a.dones)
        assert torch.equal(a.frames, frames[t]), t
        assert torch.equal(a.rewards, rewards[t]) and torch.equal(a.dones, dones[t]), t
    torch.cuda.synchronize()
    assert (a.env.get_state() == b.env.get_state()).all()
    return int(dones.sum().item())


@pytest.mark.parametrize("name,T", [("maze32_ragged", 90), ("maze6_events", 150), ("rooms16_sprites_40x48", 40),
                                    ("maze18_96x128", 45)])
def test_rollout_matches_step_sequence(name, T):
    n_done = _rollout_vs_steps(CASES[name], T, seed=13)
    if name in ("maze32_ragged", "maze18_96x128", "maze6_events"):
        assert n_done > 0


@pytest.mark.parametrize("name,T", [("maze32_ragged", 90), ("maze6_events", 150), ("ascii_coloured_rooms_shaded", 64),
                                    ("rooms16_sprites_40x48", 77)])
def test_handoff_rollout_equals_whole_env_launches(name, T):
    """A rollout of 64 or more steps runs in hand-off chunks of 12 steps that
    move between warps; shorter rollouts run each env on one warp. One chunked
    launch of T steps must equal launches of at most 32 steps covering the
    same steps, bit for bit, and leave the device error word clear."""
    cfg = CASES[name]
    N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    a, b = Run(cfg), Run(cfg)
    shape, chunk = b.env.rollout_shape(T)
    assert chunk == 12 and shape.grid <= b.env.launch_shape().grid
    assert a.env.rollout_shape(32)[1] == 0
    a.reset()
    b.reset()
    acts = torch.from_numpy(inputs.action_stream(29, T, N)).to(a.dev)
    out = []
    for run, parts in ((b, [(0, T)]), (a, [(s, min(32, T - s)) for s in range(0, T, 32)])):
        frames = torch.zeros((T, N, H, W, 3), dtype=torch.uint8, device=run.dev)
        rewards = torch.zeros((T, N), dtype=torch.float32, device=run.dev)
        dones = torch.zeros((T, N), dtype=torch.uint8, device=run.dev)
        for s, n in parts:
            run.env.rollout(acts[s:s + n], frames[s:s + n], rewards[s:s + n], dones[s:s + n])
        torch.cuda.synchronize()
        out.append((frames, rewards, dones))
    (fb, rb, db), (fa, ra, da) = out
    assert torch.equal(fa, fb) and torch.equal(ra, rb) and torch.equal(da, db)
    assert (a.env.get_state() == b.env.get_state()).all()
    b.env.sync_status()
    a.env.sync_status()


def test_handoff_rollout_replayed_in_a_cuda_graph():
    """A chunked rollout captured in a CUDA graph and replayed twice equals two
    eager launches from the same state: the hand-off counters are zeroed by
    each launch's last warp, so every replay finds them as the first did."""
    cfg = CASES["maze32_ragged"]
    N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    T = 70
    a, b = Run(cfg), Run(cfg)
    a.reset()
    b.reset()
    acts = torch.from_numpy(inputs.action_stream(31, T, N)).to(a.dev)

    def bufs(run):
        return (torch.zeros((T, N, H, W, 3), dtype=torch.uint8, device=run.dev),
                torch.zeros((T, N), dtype=torch.float32, device=run.dev),
                torch.zeros((T, N), dtype=torch.uint8, device=run.dev))

    fa, ra, da = bufs(a)
    fb, rb, db = bufs(b)
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        b.env.rollout(acts, fb, rb, db, torch.cuda.current_stream())
    torch.cuda.synchronize()
    for rep in range(2):
        a.env.rollout(acts, fa, ra, da)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(fa, fb) and torch.equal(ra, rb) and torch.equal(da, db), rep
        assert (a.env.get_state() == b.env.get_state()).all(), rep
    graph.reset()
    a.env.sync_status()
    b.env.sync_status()


def test_rollout_full_size_across_horizon():
    """4096 envs, 32 x 32 key-door mazes, in the benchmark's launch shape: a
    64-step rollout that crosses the 500-step horizon (every env resets)."""
    n_done = _rollout_vs_steps(inputs.batched_keydoor_mazes(), 64, seed=1, warm=470)
    assert n_done >= 4096


def test_envs_of_different_sizes_coexist():
    """Creating a smaller env must not break a larger one's launches (the kernel's
    shared memory limit is per function, shared by all envs of the process)."""
    big = Run(inputs.maze_keydoor(n_envs=40, map_side=32, seed=2, horizon=0, frame_h=96, frame_w=128))
    big.reset()
    small = Run(inputs.rooms(n_envs=3, map_side=8, seed=1))
    small.reset()
    for s in range(5):
        fb, _, _ = big.step(inputs.actions(1, s, 40))
        fs, _, _ = small.step(inputs.actions(2, s, 3))
    stats = Stats()
    for run in (big, small):
        ref = render_ref(run.ocfg, run.state())
        run.env.render(run.frames)
        torch.cuda.synchronize()
        compare_frames(run.frames.cpu().numpy(), ref, stats)
    stats.check()


@pytest.mark.parametrize("name,T", [("mazerooms64_gray", 60), ("mazerooms128_gray_128x128", 30)])
def test_rollout_with_gray_stack_matches_step_sequence(name, T):
    """Rollouts write the grayscale stack exactly as the step sequence does."""
    cfg = CASES[name]
    a, b = Run(cfg), Run(cfg)
    a.reset()
    b.reset()
    acts = torch.from_numpy(inputs.action_stream(19, T, cfg["n_envs"])).to(a.dev)
    N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    frames = torch.zeros((T, N, H, W, 3), dtype=torch.uint8, device=a.dev)
    rewards = torch.zeros((T, N), dtype=torch.float32, device=a.dev)
    dones = torch.zeros((T, N), dtype=torch.uint8, device=a.dev)
    b.env.rollout(acts, frames, rewards, dones)
    for t in range(T):
        a.actions.copy_(acts[t])
        a.env.step(a.actions, a.frames, a.rewards, a.dones)
        assert torch.equal(a.frames, frames[t]), t
    torch.cuda.synchronize()
    assert (a.env.get_state() == b.env.get_state()).all()  # gray planes included
    assert int(dones.sum().item()) > 0


def test_large_scale_mazes_with_rooms_sampled():
    """65,536 envs of 128 x 128 mazes with rooms, 16 sprite slots, 128 x 128 RGB and
    the grayscale stack, in the launch configuration the benchmark times (the
    batched kernel with its pinned tiling): 64 sampled envs against the oracle at
    reset, then, after rollouts up to step 496, in lockstep for 10 steps across
    the 500-step horizon, where every env takes over its pre-built next episode
    in one launch: rewards, dones, pose, turn, counters, keys, maps, regenerated
    episodes, frames, rays and grayscale stacks."""
    import bench

    cfg = inputs.large_scale()
    N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    run = Run(cfg)
    run.env.tiling = bench.parse_tiling(jx, bench.LARGE_TILING)
    stats = Stats()
    rng = np.random.default_rng(12)
    idx = np.sort(rng.choice(N, 64, replace=False))
    idx[-1] = N - 1
    run.reset()
    blob = run.env.get_state()
    gpu = to_oracle(run.env, blob, idx)
    ref = oracle.generate(run.ocfg, idx.astype(np.int32), 0, nthreads=NTHREADS)
    compare_generated(gpu, ref, run.env.S, run.env.K, "at reset")
    rr = render_ref(run.ocfg, gpu)
    compare_frames(run.frames.cpu().numpy()[idx], rr, stats)
    hits, perp = run.rays()
    compare_rays(hits[idx], perp[idx], rr, stats)
    assert (run.env.fields(blob)["gray"][idx] == oracle.gray(run.frames.cpu().numpy()[idx])[:, None]).all()
    # rollouts (4 steps per launch) up to step 496
    T, first = 4, 496
    acts = torch.from_numpy(inputs.action_stream(4, first, N)).to(run.dev)
    frames = torch.empty((T, N, H, W, 3), dtype=torch.uint8, device=run.dev)
    rewards = torch.empty((T, N), dtype=torch.float32, device=run.dev)
    dones = torch.empty((T, N), dtype=torch.uint8, device=run.dev)
    for c in range(first // T):
        run.env.rollout(acts[c * T:(c + 1) * T], frames, rewards, dones)
    torch.cuda.synchronize()
    del frames, acts
    run.env.sync_status()
    blob = run.env.get_state()
    assert (run.env.fields(blob)["t"] == first).all()
    n_reset = 0
    for s in range(first, first + 10):
        prev = to_oracle(run.env, blob, idx)
        a = inputs.actions(4, s, N)
        frames, rewards, dones = run.step(a)
        blob = run.env.get_state()
        f = run.env.fields(blob)
        cur = to_oracle(run.env, blob, idx)
        check_step(run.ocfg, idx, prev, a[idx], cur, rewards[idx], dones[idx], run.env.S, run.env.K, stats, s)
        rr = render_ref(run.ocfg, cur)
        compare_frames(frames[idx], rr, stats)
        hits, perp = run.rays()
        compare_rays(hits[idx], perp[idx], rr, stats)
        t = f["t"][idx]
        g = oracle.gray(frames[idx])
        planes = f["gray"][idx]
        assert (planes[np.arange(len(idx)), t % 4] == g).all()
        assert (planes[t == 0] == g[t == 0][:, None]).all()  # a fresh episode's frame in all four planes
        n_reset += int(dones.sum())
    assert n_reset >= N  # every env crossed the horizon
    assert (f["episode"] >= 1).all()
    run.env.sync_status()
    stats.check()


def test_pregenerated_episodes_equal_episodes_built_in_place():
    """Mazes of side >= 64 in batches large enough are built ahead by one lane
    per env (the next episode of every env whose horizon falls in the launch,
    and episode 0 at a reset); small batches build them in place, one warp per
    env. A maze depends only on (seed, env, episode), so envs 0..63 of a
    16,384-env batch and of a 64-env batch must hold the same state and give
    the same frames, rewards and dones: at the reset, and over a rollout that
    crosses the horizon (every env starts episode 1 at step 5)."""
    big_cfg = inputs.maze_rooms(n_envs=16384, map_side=64, seed=21, horizon=5, max_sprites=8, frame_h=32,
                                frame_w=32, gray_stack=0)
    small_cfg = dict(big_cfg, n_envs=64)
    big, small = Run(big_cfg), Run(small_cfg)
    big.reset()
    small.reset()
    assert torch.equal(big.frames[:64], small.frames)

    def same_state():
        fb, fs = big.env.fields(big.env.get_state()), small.env.fields(small.env.get_state())
        for name, a in fs.items():
            if name != "gray":
                assert (fb[name][:64] == a).all(), name

    same_state()
    T = 8
    acts = torch.from_numpy(inputs.action_stream(22, T, 16384)).to(big.dev)
    outs = []
    for run, n, a in ((big, 16384, acts), (small, 64, acts[:, :64].contiguous())):
        frames = torch.empty((T, n, 32, 32, 3), dtype=torch.uint8, device=run.dev)
        rewards = torch.empty((T, n), dtype=torch.float32, device=run.dev)
        dones = torch.empty((T, n), dtype=torch.uint8, device=run.dev)
        run.env.rollout(a, frames, rewards, dones)
        torch.cuda.synchronize()
        outs.append((frames, rewards, dones))
    (fb, rb, db), (fs, rs, ds) = outs
    assert int(ds.sum().item()) >= 64  # every env ended its episode (at the horizon, if not before)
    assert torch.equal(fb[:, :64], fs) and torch.equal(rb[:, :64], rs) and torch.equal(db[:, :64], ds)
    same_state()
    assert (big.env.fields(big.env.get_state())["episode"] >= 1).all()
    big.env.sync_status()
    small.env.sync_status()


def _corridor(text, n=8):
    cfg = dict(inputs.ascii_env("simple", n_envs=n, map_side=16, horizon=0), ascii_map=text)
    run = Run(cfg)
    run.reset()
    blob = run.env.get_state()
    f = run.env.fields(blob)
    f["theta0"][:] = 0.0
    f["turn"][:] = 0
    f["cell_x"][:], f["frac_x"][:] = 1, 0.45
    f["cell_y"][:], f["frac_y"][:] = 1, 0.5
    run.env.set_state(blob)
    return run


@pytest.mark.parametrize("door,passes", [("R", False), ("B", True)])
def test_coloured_key_corridor(door, passes):
    """The blue key is picked up after 16 forward moves; a red locked door then
    stops the agent at x = 4.75, a blue one lets it reach the goal after 56."""
    run = _corridor(f"#########\n#S.b.{door}.G#\n#########")
    stats = Stats()
    lockstep(run, stats, 60, seed=0, action_fn=lambda seed, step, n: np.ones(n, np.uint8))
    stats.check()
    assert stats.key_events == run.env.n
    assert stats.goal_events == (run.env.n if passes else 0)


def test_unlocked_door_opens_when_bumped():
    """Move 24 from x = 1.45 bumps the blue unlocked door at x = 4: it opens in
    the state's map; the agents then walk through, in lockstep with the oracle."""
    run = _corridor("########\n#S..\"..#\n########")
    stats = Stats()
    lockstep(run, stats, 23, seed=0, action_fn=lambda seed, step, n: np.ones(n, np.uint8))
    f = run.env.fields(run.env.get_state())
    assert (f["map"][:, 1, 4] == jx.UNLOCKED + 1).all()
    lockstep(run, stats, 1, seed=0, first_step=23, action_fn=lambda seed, step, n: np.ones(n, np.uint8))
    f = run.env.fields(run.env.get_state())
    assert (f["map"][:, 1, 4] == 0).all() and (np.abs(f["frac_x"] - 0.75) < 1e-4).all()
    lockstep(run, stats, 3, seed=0, first_step=24, action_fn=lambda seed, step, n: np.ones(n, np.uint8))
    f = run.env.fields(run.env.get_state())
    assert (f["cell_x"] == 4).all()
    stats.check()


def test_late_handoff_is_reported_and_later_rollouts_exact():
    """With the hand-off wait limit at 0 polls every hand-off of a chunked
    rollout counts as late: the launch still ends, the device error word says
    so (bit 2), and after the limit is restored and the env reset, rollouts are
    again equal to single steps (the late launch left the hand-off words clean)."""
    cfg = CASES["maze32_ragged"]
    N, H, W = cfg["n_envs"], cfg["frame_h"], cfg["frame_w"]
    T = 70
    run = Run(cfg)
    run.reset()
    acts = torch.from_numpy(inputs.action_stream(33, T, N)).to(run.dev)
    frames = torch.zeros((T, N, H, W, 3), dtype=torch.uint8, device=run.dev)
    rewards = torch.zeros((T, N), dtype=torch.float32, device=run.dev)
    dones = torch.zeros((T, N), dtype=torch.uint8, device=run.dev)
    run.env.debug_handoff_limit(0)
    run.env.rollout(acts, frames, rewards, dones)
    torch.cuda.synchronize()
    with pytest.raises(jx.JxError) as ei:
        run.env.sync_status()
    assert ei.value.status == jx.EDEVICE and "hand-off" in str(ei.value)
    run.env.debug_handoff_limit(1 << 22)
    run.env.sync_status()  # cleared by the read above
    with pytest.raises(jx.JxError):
        run.env.debug_handoff_limit(-1)
    # from a fresh reset, one chunked launch equals single steps again
    ref = Run(cfg)
    run.reset()
    ref.reset()
    run.env.rollout(acts, frames, rewards, dones)
    for t in range(T):
        ref.actions.copy_(acts[t])
        ref.env.step(ref.actions, ref.frames, ref.rewards, ref.dones)
        assert torch.equal(ref.frames, frames[t]), t
    torch.cuda.synchronize()
    assert (ref.env.get_state() == run.env.get_state()).all()
    run.env.sync_status()
