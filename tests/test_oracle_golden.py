"""Oracle pinned to hand-worked scenarios (tests/golden/*.txt).

Each scenario was worked out by hand from the rule sentences of Section IV
of the paper (cited in each file); the expected boards were not produced by
running any code.
"""
import numpy as np
import pytest

import golden_io
from oracle import OracleEnv


def _run(sc):
    env = OracleEnv([sc["H"]], [sc["W"]], [sc["mode"]], [sc["P"]], seed=7, auto_reset=0,
                    max_turns=sc["max_turns"], n_cities=0, min_general_dist=1)
    army, owner, terrain = sc["board"]
    alive = sc["alive"] if sc["alive"] is not None else (1 << sc["P"]) - 1
    env.set_game(0, army, owner, terrain, turn=sc["turn"], alive=alive)
    return env


@pytest.mark.parametrize("path", golden_io.all_scenarios(), ids=lambda p: p.split("/")[-1][:-4])
def test_golden_scenario(path):
    sc = golden_io.load(path)
    env = _run(sc)
    P = sc["P"]
    for k, step in enumerate(sc["steps"]):
        env.step(step["actions"][None, :])
        army, owner, terrain = env.board(0)
        ea, eo, et = step["board"]
        where = f"{sc['name']} step {k + 1}"
        np.testing.assert_array_equal(terrain, et, err_msg=f"terrain, {where}")
        np.testing.assert_array_equal(owner, eo, err_msg=f"owner, {where}")
        np.testing.assert_array_equal(army, ea, err_msg=f"army, {where}")
        s = env.scalars(0)
        for name, val in step["checks"].items():
            if name == "reward":
                np.testing.assert_array_equal(s["reward"][:P], np.array(val, np.float32), err_msg=where)
            else:
                assert s[name] == val, f"{name}: {s[name]} != {val}, {where}"
        for p, grids in step["obs"].items():
            ob = env.observe(0, p)
            for name, grid in grids.items():
                np.testing.assert_array_equal(ob[name].astype(np.int64), grid, err_msg=f"obs {p} {name}, {where}")
        if step["scoreboard"] is not None:
            land, arm = env.scoreboard(0)
            assert list(land[:P]) == step["scoreboard"][0]
            assert list(arm[:P]) == step["scoreboard"][1]
