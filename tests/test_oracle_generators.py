"""Pins for the oracle's map generators: spanning-tree, BFS and reachability
invariants of the key-door mazes; statistics of the random-wall rooms."""
import math

import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import breadth_first_order, connected_components, shortest_path

from paper_2605_19926_gb300 import inputs


def _grid_graph(free):
    """4-connected graph over the True cells of a 2-D mask."""
    S = free.shape[0]
    idx = np.arange(S * S).reshape(S, S)
    rows, cols = [], []
    for dy, dx in ((0, 1), (1, 0)):
        a = free[: S - dy, : S - dx] & free[dy:, dx:]
        rows += list(idx[: S - dy, : S - dx][a])
        cols += list(idx[dy:, dx:][a])
    n = S * S
    g = csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    return g + g.T


@pytest.mark.parametrize("S", [6, 8, 16, 32])
def test_maze_is_a_spanning_tree_with_keydoor_layout(orc, S):
    p = inputs.maze_keydoor(n_envs=12, map_side=S, seed=9)
    cfg = orc.make_config(**p)
    envs = orc.generate(cfg, np.arange(12), np.arange(12) % 3)
    nn = (S - 2) // 2
    types = np.bincount(np.concatenate([orc.map_view(cfg, e).reshape(-1) for e in envs]), minlength=6)[1:5]
    assert np.abs(types / types.sum() - 0.25).max() < 0.05, "wall types uniform over 1..4"
    for e in envs:
        m = orc.map_view(cfg, e).astype(int)
        assert set(np.unique(m)) <= {0, 1, 2, 3, 4, orc.DOOR}
        assert (m == orc.DOOR).sum() == 1
        assert (m[0] != 0).all() and (m[:, 0] != 0).all() and (m[S - 2:] != 0).all() and (m[:, S - 2:] != 0).all()
        open_ = m != 1
        open_ &= m != 2
        open_ &= m != 3
        open_ &= m != 4
        node = np.zeros_like(open_)
        node[1:S - 2:2, 1:S - 2:2] = True
        assert open_[node].all(), "every node is carved"
        # passages join two adjacent nodes; nothing else is open
        even_even = np.zeros_like(open_)
        even_even[0::2, 0::2] = True
        assert not (open_ & even_even).any()
        n_passages = int(open_.sum() - node.sum())
        assert n_passages == nn * nn - 1, "a spanning tree has nodes - 1 edges"
        g = _grid_graph(open_)
        ncomp, lab = connected_components(g, directed=False)
        cells = np.flatnonzero(open_.reshape(-1))
        assert len(set(lab[cells])) == 1, "connected"
        # spawn at a node centre; goal at maximal BFS distance, ties to smallest (y, x)
        sx, sy = e["x"] - 0.5, e["y"] - 0.5
        assert sx == int(sx) and sy == int(sy) and node[int(sy), int(sx)]
        s = int(sy) * S + int(sx)
        dist = shortest_path(g, indices=s, unweighted=True)
        dist[~open_.reshape(-1)] = -1
        far = dist.max()
        goal = int(np.flatnonzero(dist == far)[0])
        assert (e["goal_x"], e["goal_y"]) == (goal % S, goal // S)
        # door on the spawn-goal path at edge ceil(m/2)
        _, pred = shortest_path(g, indices=s, unweighted=True, return_predecessors=True)
        path = [goal]
        while path[-1] != s:
            path.append(int(pred[path[-1]]))
        path = path[::-1]
        mm = (len(path) - 1) // 2
        door = path[2 * ((mm + 1) // 2) - 1]
        assert (e["door_x"], e["door_y"]) == (door % S, door // S)
        assert m.reshape(-1)[door] == orc.DOOR
        # with the door closed: goal unreachable, key reachable
        closed = open_.copy()
        closed.reshape(-1)[door] = False
        reach = set(breadth_first_order(_grid_graph(closed), s, directed=False, return_predecessors=False))
        assert goal not in reach
        key = e["key_y"] * S + e["key_x"]
        assert key in reach and node.reshape(-1)[key]
        side_nodes = [c for c in reach if node.reshape(-1)[c]]
        assert key != s or len(side_nodes) == 1
        # sprites: key and goal at their cell centres
        assert e["n_sprites"] == 2
        assert (e["spr_x"][0], e["spr_y"][0], e["spr_type"][0]) == (e["key_x"] + 0.5, e["key_y"] + 0.5, 1)
        assert (e["spr_x"][1], e["spr_y"][1], e["spr_type"][1]) == (e["goal_x"] + 0.5, e["goal_y"] + 0.5, 2)
        assert 0.0 <= e["theta0"] < 2 * math.pi


def test_maze_key_is_uniform_over_spawn_side(orc):
    """Over many episodes of one maze layout family, the key lands on every
    spawn-side node with roughly equal frequency (chi-square on node counts)."""
    S = 8
    p = inputs.maze_keydoor(n_envs=1, map_side=S, seed=4)
    cfg = orc.make_config(**p)
    envs = orc.generate(cfg, np.zeros(3000, np.int32), np.arange(3000))
    # key is never on the goal side, never the spawn unless forced
    for e in envs[:200]:
        assert (e["key_x"], e["key_y"]) != (e["goal_x"], e["goal_y"])
    keys = envs["key_y"] * S + envs["key_x"]
    spawn = (envs["y"] - 0.5).astype(int) * S + (envs["x"] - 0.5).astype(int)
    assert (keys != spawn).mean() > 0.8


def test_rooms_statistics(orc):
    S = 16
    p = inputs.rooms(n_envs=200, map_side=S, wall_prob=0.25, seed=3)
    cfg = orc.make_config(**p)
    envs = orc.generate(cfg, np.arange(200))
    walls, types = 0, np.zeros(5, int)
    for e in envs:
        m = orc.map_view(cfg, e).astype(int)
        assert (m[0] > 0).all() and (m[-1] > 0).all() and (m[:, 0] > 0).all() and (m[:, -1] > 0).all()
        inner = m[1:-1, 1:-1]
        walls += (inner > 0).sum()
        types += np.bincount(m[m > 0], minlength=5)
        cx, cy = int(e["x"]), int(e["y"])
        assert m[cy, cx] == 0 and e["x"] - cx == 0.5 and e["y"] - cy == 0.5
        assert e["key_x"] == -1 and e["n_sprites"] == 0
    n = 200 * (S - 2) ** 2
    frac = walls / n
    assert abs(frac - 0.25) < 4 * math.sqrt(0.25 * 0.75 / n)
    t = types[1:] / types[1:].sum()
    assert np.abs(t - 0.25).max() < 0.02


def test_rooms_decorative_sprites_on_free_cells(orc):
    S = 16
    p = inputs.rooms(n_envs=50, map_side=S, wall_prob=0.3, seed=8, max_sprites=8)
    cfg = orc.make_config(**p)
    envs = orc.generate(cfg, np.arange(50))
    counts = envs["n_sprites"]
    assert counts.min() >= 0 and counts.max() <= 8 and len(set(counts)) > 3
    for e in envs:
        m = orc.map_view(cfg, e)
        for k in range(e["n_sprites"]):
            assert m[int(e["spr_y"][k]), int(e["spr_x"][k])] == 0
            assert e["spr_type"][k] == 3


def test_generation_is_deterministic_per_episode(orc):
    p = inputs.maze_keydoor(n_envs=4, map_side=16, seed=1)
    cfg = orc.make_config(**p)
    a = orc.generate(cfg, np.arange(4), 5)
    b = orc.generate(cfg, np.arange(4), 5)
    c = orc.generate(cfg, np.arange(4), 6)
    assert a.tobytes() == b.tobytes()
    assert (a["map"] != c["map"]).any(axis=1).all()


@pytest.mark.parametrize("S,K", [(32, 4), (64, 16), (128, 16)])
def test_maze_with_rooms_extends_the_keydoor_maze(orc, S, K):
    """The maze-with-rooms task is the key-door maze of the same seed with open
    8 x 8 squares added: the maze's floor, spawn, key, door and goal are kept;
    every added floor cell lies in an 8 x 8 window of floor (or the door) inside
    the border; all floor stays connected; sprites are key, goal, then up to
    K - 2 distractors on floor cells."""
    base = dict(inputs.maze_keydoor(n_envs=6, map_side=S, seed=17), max_sprites=K)
    c1 = orc.make_config(**base)
    c2 = orc.make_config(**dict(base, task=orc.TASK_MAZE_ROOMS))
    idx, eps = np.arange(6), np.array([0, 1, 2, 0, 5, 9])
    maze, rooms = orc.generate(c1, idx, eps), orc.generate(c2, idx, eps)
    n_added = 0
    for a, b in zip(maze, rooms):
        m1, m2 = orc.map_view(c1, a).astype(int), orc.map_view(c2, b).astype(int)
        for name in ("x", "y", "theta0", "key_x", "key_y", "goal_x", "goal_y", "door_x", "door_y"):
            assert a[name] == b[name], name
        assert (m2[m1 == 0] == 0).all(), "the maze's floor is kept"
        assert (m2 == orc.DOOR).sum() == 1 and m2[a["door_y"], a["door_x"]] == orc.DOOR
        added = (m2 == 0) & (m1 != 0)
        n_added += int(added.sum())
        open8 = (m2 == 0) | (m2 == orc.DOOR)
        # windows of 8 x 8 entirely open, by 2-D prefix sums
        ps = np.pad(open8.astype(int).cumsum(0).cumsum(1), ((1, 0), (1, 0)))
        win = ps[8:, 8:] - ps[:-8, 8:] - ps[8:, :-8] + ps[:-8, :-8] == 64
        cover = np.zeros_like(open8)
        for y0, x0 in zip(*np.nonzero(win)):
            cover[y0:y0 + 8, x0:x0 + 8] = True
        assert cover[added].all(), "added floor lies in open 8 x 8 squares"
        assert (m2[0] != 0).all() and (m2[-1] != 0).all() and (m2[:, 0] != 0).all() and (m2[:, -1] != 0).all()
        g = _grid_graph(open8)
        _, lab = connected_components(g, directed=False)
        assert len(set(lab[np.flatnonzero(open8.reshape(-1))])) == 1, "connected with the door open"
        ns = int(b["n_sprites"])
        assert 2 <= ns <= K
        assert b["spr_type"][0] == 1 and b["spr_type"][1] == 2 and (b["spr_type"][2:ns] == 3).all()
        assert (b["spr_x"][0], b["spr_y"][0]) == (b["key_x"] + 0.5, b["key_y"] + 0.5)
        for k in range(2, ns):
            assert m2[int(b["spr_y"][k]), int(b["spr_x"][k])] == 0
    if S >= 32:
        assert n_added > 0


def test_maze_with_rooms_distractor_count_is_uniform(orc):
    K = 6
    c = orc.make_config(**dict(inputs.maze_keydoor(n_envs=1, map_side=32, seed=23), max_sprites=K,
                               task=orc.TASK_MAZE_ROOMS))
    envs = orc.generate(c, np.arange(700))
    counts = np.bincount(envs["n_sprites"] - 2, minlength=K - 1)
    assert len(counts) == K - 1 and counts.min() > 0.6 * 700 / (K - 1), counts


def test_gray_is_bt601_luma(orc):
    """Integer luma: exact at black and white, and within one level of the
    real-valued BT.601 weights 0.299, 0.587, 0.114 for every RGB triple drawn."""
    rng = np.random.default_rng(3)
    rgb = rng.integers(0, 256, size=(20000, 3), dtype=np.uint8)
    rgb[:4] = [[0, 0, 0], [255, 255, 255], [255, 0, 0], [0, 255, 0]]
    g = orc.gray(rgb).astype(int)
    ref = rgb.astype(float) @ np.array([0.299, 0.587, 0.114])
    assert g[0] == 0 and g[1] == 255
    assert np.abs(g - ref).max() <= 1.0
    assert (np.diff(orc.gray(np.stack([np.arange(256)] * 3, 1).astype(np.uint8)).astype(int)) >= 0).all()
