"""Pins for the oracle's ASCII maps (Table 2 symbols), multi-colour keys and
doors, and unlocked doors, against hand-derived expectations."""
import numpy as np
import pytest

from oracle_helpers import COMMON

ALL_SYMBOLS = "\n".join([
    "##########",
    "#S.r b y #",
    "#G\"\\RBY5#",
    "#9 1 2 3 #",
    "#....G..S#",
    "##########",
])


def cfg_for(orc, text, S, max_sprites=8, **kw):
    p = dict(COMMON, task=orc.TASK_ASCII, map_side=S, frame_h=64, frame_w=64, max_sprites=max_sprites, horizon=0,
             ascii_map=text)
    p.update(kw)
    return orc.make_config(**p)


def test_symbols_map_to_cells(orc):
    """Each Table 2 symbol gives its cell: walls by colour, floor, doors by
    colour and kind; outside the text is wall."""
    S = 12
    c = cfg_for(orc, ALL_SYMBOLS, S)
    e = orc.generate(c, [0])[0]
    m = orc.map_view(c, e).astype(int)
    assert (m[0, :10] == 1).all() and (m[:, 10:] == 1).all() and (m[6:] == 1).all()
    assert list(m[1, 1:9]) == [0, 0, 0, 0, 0, 0, 0, 0]  # S . r space b space y space
    assert list(m[2, 1:9]) == [0, orc.UNLOCKED + 1, orc.UNLOCKED + 2, orc.LOCKED + 0, orc.LOCKED + 1,
                               orc.LOCKED + 2, 5, 1]  # G " \ R B Y 5 #
    assert list(m[3, 1:9]) == [9, 0, 1, 0, 2, 0, 3, 0]
    # keys in row-major order (red, blue, yellow), then the goal on one of the two G cells
    assert e["n_sprites"] == 4
    assert list(e["spr_type"][:4]) == [orc.SPR_KEY, orc.SPR_KEY_BLUE, orc.SPR_KEY_YELLOW, orc.SPR_GOAL]
    assert [(e["spr_x"][k], e["spr_y"][k]) for k in range(3)] == [(3.5, 1.5), (5.5, 1.5), (7.5, 1.5)]
    assert (e["spr_x"][3], e["spr_y"][3]) in {(1.5, 2.5), (5.5, 4.5)}
    assert (e["door_x"], e["door_y"]) == (4, 2)  # the first locked door


def test_spawn_and_goal_candidates_are_uniform(orc):
    c = cfg_for(orc, ALL_SYMBOLS, 12)
    envs = orc.generate(c, np.arange(2000))
    spawns = {(x, y) for x, y in zip(envs["x"], envs["y"])}
    assert spawns == {(1.5, 1.5), (8.5, 4.5)}
    frac = np.mean(envs["x"] == 1.5)
    assert 0.45 < frac < 0.55
    goals = envs["spr_x"][:, 3]
    assert set(goals) == {1.5, 5.5} and 0.45 < np.mean(goals == 1.5) < 0.55
    # the same env and episode always give the same episode
    again = orc.generate(c, np.arange(2000))
    assert (again["x"] == envs["x"]).all() and (again["spr_x"] == envs["spr_x"]).all()


def test_no_spawn_symbol_spawns_on_any_floor_cell(orc):
    text = "#####\n#...#\n#.#.#\n#...#\n#####"
    c = cfg_for(orc, text, 8)
    envs = orc.generate(c, np.arange(400))
    cells = {(int(x), int(y)) for x, y in zip(envs["x"], envs["y"])}
    assert cells == {(x, y) for y in (1, 2, 3) for x in (1, 2, 3) if not (x == 2 and y == 2)}


def test_bad_maps_are_rejected(orc):
    with pytest.raises(ValueError):
        orc.parse_ascii("#####\n#S..#\n#####", 4)  # too wide for S = 4
    with pytest.raises(ValueError):
        orc.parse_ascii("###\n#\t#\n###", 8)  # control character
    with pytest.raises(ValueError):
        orc.parse_ascii("###\n###", 8)  # no floor


def _walk(orc, c, e, actions):
    out = []
    for a in actions:
        r = orc.step(c, np.array([0]), e, np.array([a], np.uint8))
        out.append((float(r["rewards"][0]), int(r["dones"][0]), int(r["events"][0]), float(e["x"][0])))
    return out


def test_coloured_keys_open_only_their_doors(orc):
    """Facing +x along a corridor from x = 1.45 (x_k = 1.45 + 0.1 k): the blue
    key cell [3, 4) is entered at k = 16 (+1 reward). A red locked door at
    [5, 6) stops the box (half-size 0.2) before its right edge touches x = 5:
    move 34 would reach 4.85, so the agent stays at 4.75. With a blue door
    instead, the agent walks on and enters the goal cell [7, 8) at k = 56."""
    blocked = "#########\n#S.b.R.G#\n#########"
    open_ = "#########\n#S.b.B.G#\n#########"
    for text, passes in ((blocked, False), (open_, True)):
        c = cfg_for(orc, text, 12, step_reward=-0.001, key_reward=1.0, goal_reward=10.0)
        e = orc.generate(c, [0])
        e["theta0"] = 0.0
        e["x"] = 1.45
        res = _walk(orc, c, e, [1] * 60)
        assert not any(r[2] & orc.EV_NEAR_TIE for r in res)
        keys = [k + 1 for k, r in enumerate(res) if r[2] & orc.EV_KEY]
        goals = [k + 1 for k, r in enumerate(res) if r[2] & orc.EV_GOAL]
        assert keys == [16]
        assert np.float32(res[15][0]) == np.float32(0.999)
        if passes:
            assert goals == [56] and res[55][1] == 1
        else:
            assert goals == [] and abs(res[-1][3] - 4.75) < 1e-9


def test_unlocked_door_opens_when_bumped(orc):
    """Facing +x from x = 1.45 with a blue unlocked door at x in [4, 5): after
    23 moves the agent is at 3.75; move 24 would put the box's right edge at
    4.05, inside the door cell, so it is rejected and the door opens; moves
    25, 26, 27 then reach 3.85, 3.95, 4.05."""
    text = "########\n#S..\"..#\n########"
    c = cfg_for(orc, text, 10)
    e = orc.generate(c, [0])
    e["theta0"] = 0.0
    e["x"] = 1.45
    res = _walk(orc, c, e, [1] * 23)
    assert abs(e["x"][0] - 3.75) < 1e-9
    assert orc.map_view(c, e[0])[1, 4] == orc.UNLOCKED + 1
    res += _walk(orc, c, e, [1])
    assert abs(e["x"][0] - 3.75) < 1e-9 and orc.map_view(c, e[0])[1, 4] == 0
    res += _walk(orc, c, e, [1] * 3)
    assert abs(e["x"][0] - 4.05) < 1e-9
    assert not any(r[2] & orc.EV_NEAR_TIE for r in res)
    # a new episode starts with the door closed again
    e2 = orc.generate(c, [0], [1])
    assert orc.map_view(c, e2[0])[1, 4] == orc.UNLOCKED + 1


def test_held_key_is_not_drawn(orc):
    text = "#######\n#S.y..#\n#######"
    c = cfg_for(orc, text, 8)
    e = orc.generate(c, [0])
    e["theta0"] = 0.0
    e["x"], e["y"] = 1.5, 1.5
    yellow = np.array([232, 200, 40], np.uint8)
    f0 = orc.render(c, e)["frames"][0]
    assert (f0 == yellow).all(axis=-1).any()
    e["keys"] = 4
    f1 = orc.render(c, e)["frames"][0]
    assert not (f1 == yellow).all(axis=-1).any()
