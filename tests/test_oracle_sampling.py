"""Pins of the sampling oracle (H x W x 9 action space, Sec. IV-G; policy
head of App. C): the reproducible exponential against the library
exponential within its error bound, the expanded legal mask against the
compact observation mask and ownership, and the sampled frequencies against
the softmax of the logits (chi-square), with illegal entries never drawn."""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy import stats

from oracle import OracleEnv
from oracle.orc import exp37


def test_exp37_against_library_exp():
    xs = np.linspace(-17.3, 0.0, 20001)
    got = np.array([exp37(x) for x in xs])
    want = np.exp(xs.astype(np.float32).astype(np.float64))
    rel = np.abs(got - want) / want
    # bound: t = x log2(e) rounded to float (half an ulp of |t| <= 25 is 2^-20, i.e. 6.6e-7 relative
    # in 2^t), the Taylor tail (ln 2)^8 / 8! / 2 = 6.6e-7, Horner rounding of a few 1e-8: < 1.5e-6
    assert rel.max() < 1.5e-6, rel.max()
    assert exp37(0.0) == 1.0
    assert exp37(-30.0) == 0.0 and exp37(-17.4) == 0.0
    assert np.all(np.diff(got) >= 0)  # monotone over the grid


def _board(G=3, H=5, W=6, mode=0, P=2, seed=7, frames=12):
    env = OracleEnv(np.full(G, H), np.full(G, W), np.full(G, mode), np.full(G, P), seed=seed, n_cities=2)
    for f in range(frames):
        env.step(env.policy(100 + f))
    return env


@pytest.mark.parametrize("mode,P", [(0, 2), (1, 4), (2, 3)])
def test_mask9_matches_compact_mask_and_ownership(mode, P):
    env = _board(mode=mode, P=P)
    rng = np.random.default_rng(1)
    logits = [rng.normal(0, 2, (int(env.P[g]), 9 * int(env.N[g]))).astype(np.float32) for g in range(env.G)]
    acts, masks = env.sample_actions(logits, 5)
    for g in range(env.G):
        army, owner, terrain = env.board(g)
        for p in range(int(env.P[g])):
            ob = env.observe(g, p)
            m9 = masks[g][p].reshape(-1, 9)
            np.testing.assert_array_equal(m9[:, 0], (owner == p).astype(np.uint8))
            for k in range(1, 9):
                np.testing.assert_array_equal(m9[:, k], (ob["mask"] >> (k - 1)) & 1)
            a = acts[g, p]
            assert m9.reshape(-1)[a] == 1 or (a == 0 and not m9.any())


def _frequencies(env, logits, n_seeds):
    counts = {}
    for s in range(n_seeds):
        a, _ = env.sample_actions(logits, 1000 + s)
        counts[int(a[0, 0])] = counts.get(int(a[0, 0]), 0) + 1
    return counts


def test_sampled_frequencies_follow_softmax():
    env = _board(G=1, H=4, W=5, frames=20)
    _, masks = env.sample_actions([np.zeros((2, 9 * 20), np.float32)], 1)
    legal = np.flatnonzero(masks[0][0])
    assert legal.shape[0] >= 3
    rng = np.random.default_rng(3)
    lg = np.full((2, 9 * 20), 50.0, np.float32)  # illegal entries: large logits, never drawn
    vals = rng.choice([0.0, math.log(3.0), -1.0], size=legal.shape[0]).astype(np.float32)
    lg[0, legal] = vals
    counts = _frequencies(env, [lg], 6000)
    assert set(counts) <= set(legal.tolist())
    p = np.exp(vals.astype(np.float64))
    p /= p.sum()
    obs = np.array([counts.get(int(e), 0) for e in legal])
    chi = stats.chisquare(obs, p * obs.sum())
    assert chi.pvalue > 1e-4, (chi, obs, p)


def test_single_legal_entry_and_no_legal_entry():
    env = OracleEnv([2], [3], [0], [2], seed=1, n_cities=0, min_general_dist=1)
    army = np.array([1, 0, 0, 0, 0, 1], np.int16)
    owner = np.array([0, -1, -1, -1, -1, 1], np.int8)
    terrain = np.array([3, 0, 0, 0, 0, 3], np.int8)
    env.set_game(0, army, owner, terrain, turn=0, alive=0b01)
    lg = np.random.default_rng(0).normal(0, 5, (2, 54)).astype(np.float32)
    for s in range(20):
        a, m = env.sample_actions([lg], s)
        assert m[0][0].sum() == 1 and a[0, 0] == 0  # p0: only the pass at its general (army 1 cannot move)
    owner[5] = -1
    terrain[5] = 2
    env.set_game(0, army, owner, terrain, turn=0, alive=0b01)
    a, m = env.sample_actions([lg], 3)
    assert m[0][1].sum() == 0 and a[0, 1] == 0  # no legal entry: pass


def _one_by_three(frame=5):
    """A 1x3 board: player 0's general (5 units) | a neutral plain | player 1's
    general (5 units).  Player 0's legal entries (Q35) are, in index order,
    pass on its cell (index 0), all-but-one right (index 4) and half right
    (index 8): up, down and left leave the board."""
    env = OracleEnv(np.array([1]), np.array([3]), np.array([0]), np.array([2]), seed=1, n_cities=0,
                    min_general_dist=1)
    env.set_game(0, np.array([5, 0, 5]), np.array([0, -1, 1]), np.array([3, 0, 3]), turn=5, frame=frame)
    return env


def _logits(l0, l4, l8):
    x = np.full((2, 27), -30.0, np.float32)
    x[0, 0], x[0, 4], x[0, 8] = l0, l4, l8
    return [x]


# Worked by hand in exact integer arithmetic (Q36).  The draw of player 0 of
# game 0 at frame 5 under seed 1 is d = sm(key(1, 0, 5, 0), 7)
# = 13191151713292224422 (the hash is pinned to SplitMix64's published
# outputs in test_oracle_hash.py).
D_DRAW = 13191151713292224422


def test_sampling_worked_example_equal_weights():
    """Three legal entries of logit 0: each weighs floor(E(0) * 2^24) = 2^24,
    S = 3 * 2^24 = 50331648.  d * S = 663932404748021160745107456, whose high
    64 bits give r = 35991847.  Running sums 16777216, 33554432, 50331648:
    the first above r is the third, index 8 (half move right).  (Taking the
    low 64 bits, 14398910256543432704, exceeds S and draws nothing.)"""
    from oracle import key, sm
    assert sm(key(1, 0, 5, 0), 7) == D_DRAW
    env = _one_by_three()
    acts, masks = env.sample_actions(_logits(0.0, 0.0, 0.0), 1)
    assert masks[0][0].nonzero()[0].tolist() == [0, 4, 8]
    assert acts[0, 0] == 8


def test_sampling_worked_example_draw_on_a_boundary():
    """Weights 2^24 (pass, logit 0), 6684345 (right, logit -0.9202535152435303,
    float32 0xbf6b95bc: floor(E(x) * 2^24) = 6684345) and 0 (half right, logit
    -30 < -25 / log2 e, E = 0).  S = 23461561, d * S =
    309485010581660034102442742, r = 16777216: exactly the first running sum.
    The first entry whose running sum EXCEEDS r is the second, index 4; a
    rule of "at least r" would draw index 0, and the low 64 bits
    (760314965377661686) would draw nothing."""
    x = float(np.array([0xBF6B95BC], np.uint32).view(np.float32)[0])
    assert x == -0.9202535152435303
    assert int(np.floor(np.float32(exp37(x)) * np.float32(16777216.0))) == 6684345
    assert exp37(-30.0) == 0.0
    env = _one_by_three()
    acts, _ = env.sample_actions(_logits(0.0, x, -30.0), 1)
    assert acts[0, 0] == 4
    # one frame later the draw differs and the same weights need not pick index 4:
    # the frame is part of the key
    from oracle import key, sm
    assert sm(key(1, 0, 6, 0), 7) != D_DRAW
