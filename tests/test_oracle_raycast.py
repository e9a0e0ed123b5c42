"""Pins for the oracle's raycaster: closed forms, mirror symmetry, brute force."""
import math

import numpy as np
import pytest

from oracle_helpers import config, empty_room, env_from

H = W = 64
T30 = math.tan(math.radians(30.0))


@pytest.mark.parametrize("x0,y0", [(4.3, 8.2), (14.3, 7.9), (10.05, 6.6), (1.9, 8.0)])
def test_facing_wall_closed_form(orc, x0, y0):
    """Facing a wall at perpendicular distance d in an empty room: every column
    that hits that wall has perp = d and a slice of min(H, round(H/d)) rows."""
    S = 16
    cfg = config(S=S)
    e = env_from(S, empty_room(S), x0, y0, theta0=0.0)
    out = orc.render(cfg, e)
    rays, frame = out["rays"][0], out["frames"][0]
    d = 15.0 - x0
    h_expect = min(H, math.floor(H / d + 0.5))
    n_hit = 0
    for c in range(W):
        cx = 2.0 * (c + 0.5) / W - 1.0
        yh = y0 + d * cx * T30
        if not (1.0 + 1e-6 < yh < 15.0 - 1e-6):
            continue
        n_hit += 1
        r = rays[c]
        assert (r["cell_x"], r["side"]) == (15, 0)
        assert abs(r["perp"] - d) < 1e-12
        wall_rgb = frame[H // 2, c]
        rows = np.where((frame[:, c] == wall_rgb).all(axis=1))[0]
        assert len(rows) == h_expect
        # centred: top = floor((H - h) / 2) before clamping
        top = max(0, (H - math.floor(H / d + 0.5)) // 2)
        assert rows[0] == top
    assert n_hit > W // 2


@pytest.mark.parametrize("quarter", [1, 2, 3])
def test_facing_wall_other_headings(orc, quarter):
    """Same closed form after rotating the view by 90, 180, 270 degrees."""
    S = 16
    cfg = config(S=S)
    x0, y0 = 6.3, 9.4
    e = env_from(S, empty_room(S), x0, y0, theta0=0.0, turn=18 * quarter)
    d = {1: 15.0 - y0, 2: x0 - 1.0, 3: y0 - 1.0}[quarter]
    r = orc.render(cfg, e)["rays"][0]
    mid = r[W // 2 - 1: W // 2 + 1]
    side = 1 if quarter in (1, 3) else 0
    for ray in mid:
        assert ray["side"] == side
        assert abs(ray["perp"] - d) < 1e-9
        assert ray["h"] == math.floor(H / d + 0.5)


def _random_rooms_env(orc, rng, S=16, p=0.3, n_spr=4):
    grid = empty_room(S)
    inner = rng.random((S - 2, S - 2)) < p
    grid[1:-1, 1:-1] = np.where(inner, rng.integers(1, 5, size=inner.shape), 0)
    free = np.argwhere(grid == 0)
    y, x = free[rng.integers(len(free))]
    sprites = []
    for k in range(n_spr):
        sy, sx = free[rng.integers(len(free))]
        sprites.append((sx + 0.5, sy + 0.5, 1 + (k % 3)))
    return grid, x + rng.uniform(0.25, 0.75), y + rng.uniform(0.25, 0.75), sprites


def test_mirror_symmetry(orc):
    """Mirroring the map and pose left-right mirrors the frame column for column."""
    rng = np.random.default_rng(0)
    S = 16
    cfg = config(S=S)
    n_amb = 0
    for trial in range(40):
        grid, x, y, sprites = _random_rooms_env(orc, rng, S)
        th0 = rng.uniform(0, 2 * math.pi)
        turn = int(rng.integers(72))
        e = env_from(S, grid, x, y, th0, turn, sprites)
        em = env_from(S, grid[:, ::-1], S - x, y, math.pi - th0, (72 - turn) % 72,
                      [(S - sx, sy, st) for sx, sy, st in sprites])
        a, b = orc.render(cfg, e), orc.render(cfg, em)
        fa, fb = a["frames"][0], b["frames"][0][:, ::-1]
        amb = (a["ambiguous"][0] | b["ambiguous"][0][:, ::-1]).astype(bool)
        n_amb += amb.sum()
        diff = (fa != fb).any(axis=2)
        assert not (diff & ~amb).any(), f"trial {trial}"
        ra, rb = a["rays"][0], b["rays"][0][::-1]
        for c in range(W):
            if ra[c]["corner"] or rb[c]["corner"]:
                continue
            assert ra[c]["cell_x"] == S - 1 - rb[c]["cell_x"]
            assert ra[c]["cell_y"] == rb[c]["cell_y"] and ra[c]["side"] == rb[c]["side"]
            assert abs(ra[c]["perp"] - rb[c]["perp"]) <= 1e-12 * ra[c]["perp"]
    assert n_amb < 0.001 * 40 * H * W


def _march(grid, ox, oy, dx, dy, dt=1e-4, tmax=16.0):
    """Fine-step marching: first sample inside a solid cell; side from which
    cell index changed; None when both changed in one step (a corner)."""
    S = grid.shape[0]
    t = np.arange(0.0, tmax, dt)
    px, py = ox + t * dx, oy + t * dy
    cx, cy = np.floor(px).astype(int), np.floor(py).astype(int)
    inside = (cx >= 0) & (cy >= 0) & (cx < S) & (cy < S)
    solid = np.ones_like(inside)
    solid[inside] = grid[cy[inside], cx[inside]] != 0
    k = int(np.argmax(solid))
    assert solid[k] and k > 0
    chx, chy = cx[k] != cx[k - 1], cy[k] != cy[k - 1]
    if chx and chy:
        return None
    return cx[k], cy[k], (0 if chx else 1), t[k]


def test_dda_matches_brute_force_marching(orc):
    rng = np.random.default_rng(1)
    S = 8
    cfg = config(S=S)
    checked = 0
    for _ in range(150):
        grid = empty_room(S)
        grid[1:-1, 1:-1] = (rng.random((S - 2, S - 2)) < 0.3).astype(np.uint8) * 2
        free = np.argwhere(grid == 0)
        if len(free) == 0:
            continue
        y, x = free[rng.integers(len(free))]
        ox, oy = x + rng.uniform(0.05, 0.95), y + rng.uniform(0.05, 0.95)
        a = rng.uniform(0, 2 * math.pi)
        dx, dy = math.cos(a), math.sin(a)
        e = env_from(S, grid, ox, oy)
        m = _march(grid, ox, oy, dx, dy)
        if m is None:
            continue
        r = orc.cast(cfg, e, ox, oy, dx, dy)
        assert (r["cell_x"], r["cell_y"], r["side"]) == m[:3]
        assert m[3] - 1e-4 - 1e-9 <= r["perp"] <= m[3] + 1e-9
        checked += 1
    assert checked > 120


def test_sprite_straight_ahead_closed_form(orc):
    """A goal sprite straight ahead at depth D spans the pixel centres inside
    [W/2 - hw, W/2 + hw) x [H/2, H/2 + H/(2D)), hw = (W/2) 0.25 / (tan30 D)."""
    S = 16
    cfg = config(S=S)
    for D in (1.3, 2.0, 4.0, 7.25):
        e = env_from(S, empty_room(S), 3.5, 8.5, 0.0, 0, sprites=[(3.5 + D, 8.5, 2)])
        frame = orc.render(cfg, e)["frames"][0]
        goal = (frame == np.array([240, 208, 32], np.uint8)).all(axis=2)
        hw = 0.5 * W * 0.25 / (T30 * D)
        cols = [c for c in range(W) if W / 2 - hw <= c + 0.5 < W / 2 + hw]
        rows = [r for r in range(H) if H / 2 <= r + 0.5 < H / 2 + H / (2 * D)]
        expect = np.zeros((H, W), bool)
        expect[np.ix_(rows, cols)] = True
        assert (goal == expect).all(), D


def test_sprite_off_axis_and_occlusion(orc):
    S = 16
    cfg = config(S=S)
    D, L = 5.0, 1.0
    e = env_from(S, empty_room(S), 3.5, 7.5, 0.0, 0, sprites=[(3.5 + D, 7.5 + L, 2)])
    goal = (orc.render(cfg, e)["frames"][0] == np.array([240, 208, 32], np.uint8)).all(axis=2)
    cols = np.where(goal.any(axis=0))[0]
    centre = 0.5 * W * (1 + (L / T30) / D)
    assert abs((cols[0] + cols[-1] + 1) / 2 - centre) <= 1.0
    # a wall cell between the agent and the sprite hides it
    grid = empty_room(S)
    grid[7, 5] = 3
    grid[8, 5] = 3
    e2 = env_from(S, grid, 3.5, 7.5, 0.0, 0, sprites=[(3.5 + D, 7.5 + L, 2)])
    goal2 = (orc.render(cfg, e2)["frames"][0] == np.array([240, 208, 32], np.uint8)).all(axis=2)
    assert not goal2.any()


def test_sprite_mask_areas(orc):
    """Key (diamond) covers ~1/2 of its rectangle, a distractor (disc) ~pi/4."""
    S = 16
    cfg = config(S=S, H=128, W=128)
    areas = {}
    for st in (1, 2, 3):
        e = env_from(S, empty_room(S), 3.5, 8.5, 0.0, 0, sprites=[(4.6, 8.5, st)])
        f = orc.render(cfg, e)["frames"][0]
        colours = {1: [224, 40, 40], 2: [240, 208, 32], 3: [144, 64, 192]}
        areas[st] = (f == np.array(colours[st], np.uint8)).all(axis=2).sum()
    assert abs(areas[1] / areas[2] - 0.5) < 0.03
    assert abs(areas[3] / areas[2] - math.pi / 4) < 0.03


def test_locked_door_blocks_rays_until_key(orc):
    S = 16
    cfg = config(task=1, S=S)
    grid = empty_room(S)
    grid[:, 8] = 2
    grid[8, 8] = orc.DOOR
    e = env_from(S, grid, 4.5, 8.5, 0.0)
    r = orc.render(cfg, e)["rays"][0][W // 2]
    assert (r["cell_x"], r["cell_y"]) == (8, 8)
    e["keys"] = 1
    r = orc.render(cfg, e)["rays"][0][W // 2]
    assert r["cell_x"] == 15


def test_screen_handedness(orc):
    """With the map's y axis pointing down and the heading measured from +x
    towards +y, the screen's left edge looks towards -y: facing +x next to the
    top wall, column 0 hits the top wall and column W-1 the right wall."""
    S = 16
    cfg = config(S=S)
    grid = empty_room(S)
    e = env_from(S, grid, 2.5, 1.5, 0.0)
    rays = orc.render(cfg, e)["rays"][0]
    assert (rays[0]["cell_y"], rays[0]["side"]) == (0, 1)
    assert (rays[W - 1]["cell_x"], rays[W - 1]["side"]) == (15, 0)


@pytest.mark.parametrize("d", [0.8, 1.0, 2.0, 4.0, 7.5, 13.0])
def test_distance_shading_closed_form(orc, d):
    """Distance shading facing a wall at distance d (x face, type-1 wall of RGB
    (160, 160, 160)): the slice of h = min(H, round(H/d)) rows is drawn at
    160 q / 256 per channel, q = 64 + floor(192 min(h, H) / H) -- full colour
    at d <= 1, 160 * 160 / 256 = 100 at d = 2, tending to a quarter far away --
    and the unshaded frame differs only in the wall's colour."""
    S = 16
    x0, y0 = 15.0 - d, 8.2
    plain = orc.render(config(S=S), env_from(S, empty_room(S), x0, y0, theta0=0.0))["frames"][0]
    shaded = orc.render(config(S=S, shading=1), env_from(S, empty_room(S), x0, y0, theta0=0.0))["frames"][0]
    h = min(H, math.floor(H / d + 0.5))
    q = 64 + (192 * h) // H
    c = W // 2
    col_p, col_s = plain[:, c], shaded[:, c]
    wall = (col_p == np.array([160, 160, 160], np.uint8)).all(axis=1)
    assert wall.sum() == h
    assert (col_s[wall] == (160 * q) >> 8).all()
    assert (col_s[~wall] == col_p[~wall]).all()
    if d <= 1.0:
        assert (col_s[wall] == 160).all()
    if d == 2.0:
        assert (col_s[wall] == 100).all()
    assert (col_s[wall] >= 40).all()


def test_distance_shading_is_monotone(orc):
    """Nearer walls are never darker than farther ones."""
    S = 16
    vals = []
    for d in (0.6, 1.5, 2.5, 3.5, 5.0, 8.0, 12.0):
        f = orc.render(config(S=S, shading=1), env_from(S, empty_room(S), 15.0 - d, 8.2, theta0=0.0))["frames"][0]
        vals.append(int(f[H // 2, W // 2, 0]))
    assert all(a >= b for a, b in zip(vals, vals[1:])), vals
    assert vals[0] == 160 and vals[-1] < 160
