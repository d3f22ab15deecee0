"""Pins of the feature-tensor oracle (Appendix A, table of observation channels).

* Hand-worked scenarios (tests/golden/features/): selected channels after each
  step, derived by hand from the table and the readings Q26-Q33.
* Invariants over random rollouts in every mode, checked against the
  oracle's observation, board and scoreboard (separate functions of the rule
  oracle): the ownership partition of each cell, the instantaneous army rows,
  fog = 1 - visibility, persistent masks growing within an episode and
  cleared by a new one, the last-seen enemy army on visible cells, the age
  row taking values log(1 + dt) / 5 for integer dt <= turn, and the delta
  rows against the army planes the test records itself.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

from golden_io import parse_board, parse_mode, action_index
from oracle.orc import OracleEnv, OracleFeatures

FEAT_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "features")


def load_feature_case(path):
    lines = [ln.rstrip() for ln in open(path)]
    lines = [ln for ln in lines if ln.strip() and not ln.lstrip().startswith("#")]
    sc = {"frames": []}
    i = 0
    H = W = None
    while i < len(lines):
        t = lines[i].split()
        if t[0] == "mode":
            sc["mode"], sc["P"] = parse_mode(t[1])
            i += 1
        elif t[0] == "size":
            H, W = int(t[1]), int(t[2])
            sc["H"], sc["W"] = H, W
            i += 1
        elif t[0] == "turn":
            sc["turn"] = int(t[1])
            i += 1
        elif t[0] == "hist":
            sc["hist"] = int(t[1])
            i += 1
        elif t[0] == "window":
            sc["window"] = int(t[1])
            i += 1
        elif t[0] == "series":
            sc["frames"][-1]["series"].append(tuple(int(x) for x in t[1:5]))
            i += 1
        elif t[0] == "board":
            sc["board"] = parse_board(lines[i + 1:i + 1 + H], H, W)
            i += 1 + H
        elif t[0] == "frame":
            sc["frames"].append({"actions": None, "checks": [], "series": []})
            i += 1
        elif t[0] == "step":
            acts = np.zeros(8, np.int32)
            i += 1
            for _ in range(sc["P"]):
                p, a = action_index(lines[i], W)
                acts[p] = a
                i += 1
            sc["frames"].append({"actions": acts, "checks": [], "series": []})
        elif t[0] == "ch":
            grid = np.array([[float(x) for x in ln.split()] for ln in lines[i + 1:i + 1 + H]]).reshape(-1)
            sc["frames"][-1]["checks"].append((int(t[1]), int(t[2]), grid))
            i += 1 + H
        elif t[0] == "scalar":
            sc["frames"][-1]["checks"].append((int(t[1]), int(t[2]), np.full(H * W, float(t[3]))))
            i += 1
        else:
            raise ValueError(f"{path}: unknown line {lines[i]!r}")
    return sc


def feature_cases():
    return sorted(f for f in os.listdir(FEAT_DIR) if f.endswith(".txt") and f != "README.txt")


@pytest.mark.parametrize("name", feature_cases())
def test_feature_golden(name):
    sc = load_feature_case(os.path.join(FEAT_DIR, name))
    env = OracleEnv([sc["H"]], [sc["W"]], [sc["mode"]], [sc["P"]], auto_reset=0)
    army, owner, terrain = sc["board"]
    env.set_game(0, army, owner, terrain, turn=sc["turn"])
    fb = OracleFeatures(env, hist=sc["hist"], window=sc.get("window", 0))
    n_checks = 0
    for k, fr in enumerate(sc["frames"]):
        if fr["actions"] is not None:
            env.step(fr["actions"][None, :])
        feats = fb.build()[0]
        assert feats.shape == (sc["P"], 24 + 2 * sc["hist"], sc["H"] * sc["W"])
        for p, ch, want in fr["checks"]:
            got = feats[p, ch].astype(np.float64)
            np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-9,
                                       err_msg=f"{name}: frame {k} player {p} channel {ch}")
            n_checks += 1
        for p, k, army, land in fr["series"]:
            assert tuple(fb.series[0][p, k]) == (army, land), (name, k, p, fb.series[0][p, k])
            n_checks += 1
    assert n_checks > 10


def test_feature_build_is_idempotent_within_a_frame():
    env = OracleEnv([7], [9], [0], [2], seed=11)
    fb = OracleFeatures(env, hist=3)
    rng = np.random.default_rng(0)
    for _ in range(5):
        env.step(env.policy(int(rng.integers(1 << 30))))
        a = fb.build()[0].copy()
        b = fb.build()[0]
        np.testing.assert_array_equal(a, b)


def _team(mode, q):
    return q >> 1 if mode == 1 else q


@pytest.mark.parametrize("mode,P,side", [(0, 2, (6, 11)), (1, 4, (7, 12)), (2, 5, (8, 12))])
def test_feature_invariants(mode, P, side):
    rng = np.random.default_rng(100 + mode)
    G = 4
    H = rng.integers(side[0], side[1] + 1, G)
    W = rng.integers(side[0], side[1] + 1, G)
    hist, window = 4, 16
    env = OracleEnv(H, W, np.full(G, mode), np.full(G, P), seed=5 + mode, n_cities=3, max_turns=37)
    fb = OracleFeatures(env, hist=hist, window=window)
    series = {}      # (g, p) -> recorded (opponents' army, land), newest first
    own_hist = {}    # (g, p) -> planes, newest first, of this episode
    enemy_hist = {}
    prev = {}
    epochs = [env.scalars(g)["epoch"] for g in range(G)]
    resets_seen = 0
    for t in range(90):
        if t:
            env.step(env.policy(1000 + t))
        feats = fb.build()
        for g in range(G):
            sc = env.scalars(g)
            if sc["epoch"] != epochs[g]:
                resets_seen += 1
                epochs[g] = sc["epoch"]
                for p in range(P):
                    own_hist.pop((g, p), None)
                    enemy_hist.pop((g, p), None)
                    series.pop((g, p), None)
                    prev.pop((g, p), None)
            army, owner, terrain = env.board(g)
            land, tot = env.scoreboard(g)
            N = int(H[g] * W[g])
            for p in range(P):
                f = feats[g][p].astype(np.float64)
                ob = env.observe(g, p)
                vis = ob["vis"].astype(bool)
                opp = np.array([o >= 0 and _team(mode, o) != _team(mode, p) for o in owner])
                ally = np.array([o >= 0 and o != p and _team(mode, o) == _team(mode, p) for o in owner])
                mtn = terrain == 1
                # instantaneous rows
                np.testing.assert_array_equal(f[12], (~vis).astype(float))
                np.testing.assert_array_equal(f[10], (owner == p).astype(float))
                part = f[9] + f[10] + f[11] + f[12] + (vis & mtn) + (vis & ally)
                np.testing.assert_array_equal(part, np.ones(N))
                np.testing.assert_array_equal(f[0], np.where(vis, army, 0))
                np.testing.assert_array_equal(f[0], f[1] + f[2] + f[3] + np.where(vis & ally, army, 0))
                assert np.all(f[13] <= f[12])
                # scoreboard rows
                oppq = [q for q in range(P) if _team(mode, q) != _team(mode, p)]
                assert f[16][0] == land[p] and f[17][0] == tot[p]
                assert f[18][0] == sum(land[q] for q in oppq) and f[19][0] == sum(tot[q] for q in oppq)
                assert np.all(f[14] == sc["turn"])
                # temporal tokens: this frame's opponents' totals first, then the recorded past, zeros before
                rec = [(sum(tot[q] for q in oppq), sum(land[q] for q in oppq))] + series.get((g, p), [])
                series[(g, p)] = rec[:window]
                want = np.zeros((window, 2), np.int64)
                want[:len(series[(g, p)])] = series[(g, p)]
                np.testing.assert_array_equal(fb.series[g][p], want)
                # memory
                assert np.all(f[4] >= vis)
                assert np.all(f[5] >= (vis & opp))
                for ch, code in ((6, 3), (7, 2), (8, 1)):  # generals, castles, mountains in sight
                    assert np.all(f[ch] >= (vis & (terrain == code))), ch
                np.testing.assert_array_equal(f[20][vis], f[2][vis])
                if (g, p) in prev:
                    for ch in (4, 5, 6, 7, 8):
                        assert np.all(f[ch] >= prev[(g, p)][ch]), ch
                else:
                    np.testing.assert_array_equal(f[4], vis.astype(float))
                dt = np.expm1(5.0 * f[21])
                assert np.allclose(dt, np.round(dt), atol=1e-3)
                assert np.all(np.round(dt) <= sc["turn"]) and np.all(f[21][vis] == 0)
                prev[(g, p)] = f
                # delta rows against recorded planes
                own = np.where(owner == p, army, 0).astype(np.int64)
                enemy = np.where(vis & opp, army, 0).astype(np.int64)
                oh = [own] + own_hist.get((g, p), [])
                eh = [enemy] + enemy_hist.get((g, p), [])
                own_hist[(g, p)], enemy_hist[(g, p)] = oh[:hist + 1], eh[:hist + 1]
                z = np.zeros(N, np.int64)
                for k in range(hist):
                    a0, a1 = (oh + [z] * (hist + 2))[k], (oh + [z] * (hist + 2))[k + 1]
                    e0, e1 = (eh + [z] * (hist + 2))[k], (eh + [z] * (hist + 2))[k + 1]
                    np.testing.assert_array_equal(f[24 + k], a0 - a1)
                    np.testing.assert_array_equal(f[24 + hist + k], e0 - e1)
    assert resets_seen >= 1
