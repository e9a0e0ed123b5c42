"""Pins for the oracle's tie-biased step and render: the outcomes a
finite-precision tie admits. Where a collision, pickup or DDA decision lies
within the tie tolerance, each biased variant must give one definite side of
it (closed forms on hand-built cases); where no decision is that close, every
variant must equal the exact step or frame."""
import itertools
import math

import numpy as np

import oracle
from oracle_helpers import config, empty_room, env_from

VARIANTS = list(itertools.product((-1, 1), (-1, 1), (-1, 1), (-1, 1)))


def test_collision_tie_both_outcomes(orc):
    """A box whose edge lands exactly on a wall face: touching blocks (the
    exact test), a box smaller by the tolerance moves. Bias +1 takes the move,
    bias -1 the block, and the step is flagged as a near tie."""
    S = 8
    grid = empty_room(S)
    grid[1:-1, 6] = 2  # a wall column at x = 6
    cfg = config(S=S)
    # edge at x + 0.1 + 0.2: at 5.7 it ends on the face x = 6 (to rounding)
    out = {}
    for bias in (0, 1, -1):
        e = env_from(S, grid, 5.7, 3.5, 0.0, 0)
        o = orc.step_biased(cfg, np.array([0]), e, np.array([1], np.uint8), bias, 0, 0, 0)
        assert o["events"][0] & oracle.EV_NEAR_TIE
        out[bias] = float(e["x"][0])
    assert math.isclose(out[1], 5.8, abs_tol=1e-12)  # moved
    assert out[-1] == 5.7  # blocked
    assert out[0] in (out[1], out[-1])


def test_pickup_tie_both_outcomes(orc):
    """An agent 1e-7 cells left of the key's cell: the exact test misses the
    key, the test point moved right by the tolerance picks it up."""
    S = 8
    cfg = config(S=S)
    spr = [(5.5, 3.5, oracle.SPR_KEY)]
    got = {}
    for px in (-1, 0, 1):
        e = env_from(S, empty_room(S), 5.0 - 1e-7, 3.5, 0.0, 0, sprites=spr, key=(5, 3))
        o = orc.step_biased(cfg, np.array([0]), e, np.array([0], np.uint8), 0, 0, px, 0)
        assert o["events"][0] & oracle.EV_NEAR_TIE
        got[px] = (float(o["rewards"][0]), int(e["keys"][0]))
    assert got[1] == (np.float32(-0.001 + 1.0), 1)
    assert got[-1] == (np.float32(-0.001), 0) and got[0] == got[-1]


def test_variants_equal_exact_step_without_ties(orc):
    """Away from ties every biased variant is the exact step (rewards, dones,
    poses, keys, regenerated episodes)."""
    cfg = orc.make_config(task=1, map_side=16, frame_h=32, frame_w=32, max_sprites=2, horizon=6, turns_per_rev=72,
                          fov_deg=60.0, move_step=0.1, radius=0.2, step_reward=-0.001, key_reward=1.0,
                          goal_reward=10.0, seed=11)
    n = 64
    idx = np.arange(n, dtype=np.int32)
    envs = orc.generate(cfg, idx)
    rng = np.random.default_rng(3)
    checked = 0
    for s in range(8):
        a = rng.integers(0, 7, size=n, dtype=np.uint8)
        exact = envs.copy()
        ref = orc.step(cfg, idx, exact, a)
        clean = (ref["events"] & oracle.EV_NEAR_TIE) == 0
        for v in VARIANTS:
            var = envs.copy()
            o = orc.step_biased(cfg, idx, var, a, *v)
            assert (o["rewards"][clean] == ref["rewards"][clean]).all()
            assert (o["dones"][clean] == ref["dones"][clean]).all()
            assert (var[clean] == exact[clean]).all()
        checked += int(clean.sum())
        envs = exact
    assert checked > 400


def _corner_env(S=8):
    """Agent at (2.5, 2.5) looking along the diagonal through the lattice
    point (3, 3); walls at its x neighbour (3, 2) (type 2) and its y
    neighbour (2, 3) (type 3)."""
    grid = empty_room(S)
    grid[2, 3] = 2
    grid[3, 2] = 3
    return grid


def test_cast_corner_bias(orc):
    S = 8
    cfg = config(S=S)
    e = env_from(S, _corner_env(S), 2.5, 2.5)
    r0 = orc.cast(cfg, e, 2.5, 2.5, 1.0, 1.0, 0)
    rx = orc.cast(cfg, e, 2.5, 2.5, 1.0, 1.0, 1)
    ry = orc.cast(cfg, e, 2.5, 2.5, 1.0, 1.0, -1)
    assert (rx["cell_x"], rx["cell_y"], rx["side"]) == (3, 2, 0)
    assert (ry["cell_x"], ry["cell_y"], ry["side"]) == (2, 3, 1)
    assert (r0["cell_x"], r0["cell_y"], r0["side"]) == (2, 3, 1)  # exact tie: y on "not strictly less"
    assert rx["perp"] == ry["perp"] == 0.5


def test_biased_render_draws_each_corner_decision(orc):
    """A column whose ray passes through a lattice point: the +1 frame draws
    the x neighbour's x face at full colour, the -1 frame the y neighbour's
    y face at 3/4; both equal the exact frame in every other column, and
    neither flags the corner column as wholly ambiguous."""
    S, H, W = 8, 64, 64
    cfg = config(S=S, H=H, W=W)
    T = math.tan(math.radians(30.0))
    col = 20
    cx = 2.0 * (col + 0.5) / W - 1.0
    th = math.pi / 4
    rx, ry = math.cos(th) - cx * T * math.sin(th), math.sin(th) + cx * T * math.cos(th)
    ox, oy = 3.0 - 0.5 * rx, 3.0 - 0.5 * ry  # the column's ray meets (3, 3) at t = 0.5
    grid = _corner_env(S)
    e = env_from(S, grid, ox, oy, th, 0)
    assert math.floor(ox) == 2 and math.floor(oy) == 2
    ex = orc.render(cfg, e)
    assert ex["rays"]["corner"][0, col] == 1
    fx, fy = orc.render(cfg, e, bias=1), orc.render(cfg, e, bias=-1)
    assert (fx["rays"]["cell_x"][0, col], fx["rays"]["cell_y"][0, col], fx["rays"]["side"][0, col]) == (3, 2, 0)
    assert (fy["rays"]["cell_x"][0, col], fy["rays"]["cell_y"][0, col], fy["rays"]["side"][0, col]) == (2, 3, 1)
    other = [c for c in range(W) if not ex["rays"]["corner"][0, c]]
    for f in (fx, fy):
        assert (f["frames"][0][:, other] == ex["frames"][0][:, other]).all()
        assert f["ambiguous"][0][:, col].sum() <= 4
    mid = H // 2
    wall2, wall3 = fx["frames"][0, mid, col], fy["frames"][0, mid, col]
    ref2 = orc.render(cfg, env_from(S, empty_room(S, wall=2), 3.5, 3.5, 0.0, 0))["frames"][0, mid, W // 2]
    ref3 = orc.render(cfg, env_from(S, empty_room(S, wall=3), 3.5, 3.5, math.pi / 2, 0))["frames"][0, mid, W // 2]
    assert (wall2 == ref2).all()  # x face of wall type 2, full colour (facing +x)
    assert (wall3 == ref3).all()  # y face of wall type 3, 3/4 colour (facing +y)
