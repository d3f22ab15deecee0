"""Oracle pinned to closed forms, library routines, brute force and invariants.

* growth under all-pass play: general army at turn t is 1 + floor(t/2), an
  owned plain cell gains floor(t/50), an owned castle floor(t/2) (Sec. IV-C);
* fog equals a 3x3 binary dilation of the (team) ownership mask computed by
  scipy.ndimage (Sec. IV-B: own cells plus their Moore neighbourhood);
* the mask bit of every one of the 8 move kinds equals whether the step
  itself executes that action alone (checked through the invalid counter);
* generator: mountain share, castle count and army range, general spacing,
  4-connectivity of all generals (scipy.ndimage.label) (Sec. IV-A);
* benchmark policy: always legal, uniform over legal pairs (chi-square),
  split rate 0.2;
* invariants on random rollouts of every mode and exhaustively over joint
  actions on 3x3 boards: owner range, neutral zero-army mountains, alive
  players hold their generals, the dead hold nothing, army change minus
  growth is a non-positive even number when no general falls.
"""
import itertools

import numpy as np
import pytest
from scipy import ndimage

from oracle import OracleEnv
from paper_2606_23348_gb300.workloads import shapes

T_PLAIN, T_MTN, T_CASTLE, T_GEN = 0, 1, 2, 3
SPLIT = 858993459


def make_env(G, H, W, mode=0, n_players=2, **kw):
    Hs = np.full(G, H, np.int32) if np.isscalar(H) else np.asarray(H, np.int32)
    Ws = np.full(G, W, np.int32) if np.isscalar(W) else np.asarray(W, np.int32)
    ms = np.full(G, mode, np.int32) if np.isscalar(mode) else np.asarray(mode, np.int32)
    ps = np.full(G, n_players, np.int32) if np.isscalar(n_players) else np.asarray(n_players, np.int32)
    kw.setdefault("n_cities", 8)
    return OracleEnv(Hs, Ws, ms, ps, **kw)


# ---------------------------------------------------------------- growth
def test_growth_closed_form_all_pass():
    H = W = 6
    env = make_env(1, H, W, auto_reset=0)
    army = np.zeros(H * W, np.int16)
    owner = np.full(H * W, -1, np.int8)
    terrain = np.zeros(H * W, np.int8)
    terrain[0], owner[0], army[0] = T_GEN, 0, 1
    terrain[35], owner[35], army[35] = T_GEN, 1, 1
    terrain[7], owner[7], army[7] = T_CASTLE, 0, 3
    terrain[8], army[8] = T_CASTLE, 44          # neutral castle: never grows
    owner[14], army[14] = 1, 5                  # owned plain
    owner[20], army[20] = 0, 0
    env.set_game(0, army, owner, terrain, turn=0)
    for t in range(1, 161):
        env.step(np.zeros((1, 2), np.int32))
        a, o, _ = env.board(0)
        assert a[0] == 1 + t // 2 and a[35] == 1 + t // 2
        assert a[7] == 3 + t // 2
        assert a[8] == 44
        assert a[14] == 5 + t // 50 and a[20] == t // 50
        assert env.scalars(0)["turn"] == t


# ---------------------------------------------------------------- fog, obs
def _random_state(rng, H, W, P, mode):
    N = H * W
    terrain = np.where(rng.random(N) < 0.2, T_MTN, T_PLAIN).astype(np.int8)
    owner = np.full(N, -1, np.int8)
    army = np.zeros(N, np.int16)
    cells = rng.permutation(N)
    gens = cells[:P]
    for p, c in enumerate(gens):
        terrain[c], owner[c], army[c] = T_GEN, p, rng.integers(1, 30)
    for c in cells[P:P + 3]:
        if terrain[c] == T_PLAIN:
            terrain[c], army[c] = T_CASTLE, rng.integers(0, 50)
    free = [c for c in range(N) if terrain[c] != T_MTN and terrain[c] != T_GEN]
    for c in free:
        if rng.random() < 0.4:
            owner[c] = rng.integers(0, P)
            army[c] = rng.integers(0, 12)
        elif terrain[c] == T_PLAIN and rng.random() < 0.2:
            army[c] = rng.integers(0, 3)
    return army, owner, terrain


@pytest.mark.parametrize("mode,P", [(0, 2), (1, 4), (2, 5)])
def test_fog_equals_binary_dilation(mode, P):
    rng = np.random.default_rng(11 + mode)
    H, W = 7, 9
    env = make_env(1, H, W, mode, P, auto_reset=0)
    for trial in range(25):
        army, owner, terrain = _random_state(rng, H, W, P, mode)
        alive = int(rng.integers(0, 1 << P)) | 1
        env.set_game(0, army, owner, terrain, turn=3, alive=alive)
        for p in range(P):
            ob = env.observe(0, p)
            team = [q for q in range(P) if (q >> 1 if mode == 1 else q) == (p >> 1 if mode == 1 else p)]
            mine = np.isin(owner, team).reshape(H, W)
            want = ndimage.binary_dilation(mine, structure=np.ones((3, 3), bool)).reshape(-1)
            if not (alive >> p) & 1:
                want[:] = False
            np.testing.assert_array_equal(ob["vis"].astype(bool), want)
            v = want
            np.testing.assert_array_equal(ob["army"], np.where(v, army, 0))
            np.testing.assert_array_equal(ob["owner"], np.where(v, owner, -2))
            fogged = np.where(np.isin(terrain, [T_MTN, T_CASTLE]), 5, 4)
            np.testing.assert_array_equal(ob["terrain"], np.where(v, terrain, fogged))


@pytest.mark.parametrize("mode,P", [(0, 2), (1, 4), (2, 3)])
def test_mask_equals_step_validator(mode, P):
    """Every mask bit is checked by executing that single action in the step."""
    rng = np.random.default_rng(5 + mode)
    H, W = 4, 5
    N = H * W
    env = make_env(1, H, W, mode, P, auto_reset=0)
    for trial in range(6):
        army, owner, terrain = _random_state(rng, H, W, P, mode)
        alive = (1 << P) - 1
        if trial % 3 == 2:
            alive &= ~2  # one player out
        for p in range(P):
            env.set_game(0, army, owner, terrain, turn=p, alive=alive)  # p moves first
            mask = env.observe(0, p)["mask"]
            for c in range(N):
                for k in range(1, 9):
                    env.set_game(0, army, owner, terrain, turn=p, alive=alive)
                    before = env.scalars(0)["invalid"]
                    acts = np.zeros((1, P), np.int32)
                    acts[0, p] = c * 9 + k
                    env.step(acts)
                    executed = env.scalars(0)["invalid"] == before
                    if not (alive >> p) & 1:
                        executed = False  # a dead player's action is skipped, never executed
                    bit = (k - 1) if k <= 4 else (4 + k - 5)
                    assert bool((mask[c] >> bit) & 1) == executed, (trial, p, c, k)


def test_scoreboard_recount():
    rng = np.random.default_rng(3)
    env = make_env(1, 6, 6, 2, 4, auto_reset=0)
    army, owner, terrain = _random_state(rng, 6, 6, 4, 2)
    env.set_game(0, army, owner, terrain)
    land, arm = env.scoreboard(0)
    for p in range(4):
        assert land[p] == int((owner == p).sum())
        assert arm[p] == int(army[owner == p].astype(np.int64).sum())


# ---------------------------------------------------------------- generator
def test_generator_statistics_15x15():
    G = 400
    env = make_env(G, 15, 15, auto_reset=0, seed=1, n_cities=8, min_general_dist=0)
    mfrac, armies = [], []
    for g in range(G):
        a, o, t = env.board(g)
        s = env.scalars(g)
        mfrac.append(float((t == T_MTN).mean()))
        cas = t == T_CASTLE
        assert cas.sum() == 8
        assert np.all(o[cas] == -1)
        armies.extend(a[cas].tolist())
        gens = np.flatnonzero(t == T_GEN)
        assert len(gens) == 2
        assert sorted(o[gens].tolist()) == [0, 1] and np.all(a[gens] == 1)
        (r0, c0), (r1, c1) = divmod(s["gpos"][0], 15), divmod(s["gpos"][1], 15)
        assert abs(r0 - r1) + abs(c0 - c1) >= 10  # floor((15 + 15) / 3)
        assert np.all(a[(t == T_MTN)] == 0) and np.all(o[t == T_MTN] == -1)
        assert np.all(o[(t != T_GEN)] == -1)
        lab, _ = ndimage.label((t != T_MTN).reshape(15, 15))
        assert lab.reshape(-1)[gens[0]] == lab.reshape(-1)[gens[1]]
        assert s["turn"] == 0 and s["epoch"] == 0 and s["alive"] == 3
    m = float(np.mean(mfrac))
    # raw Bernoulli share is 0.2; the carved path (<= 28 cells) lowers it
    assert 0.2 - 30 / 225 < m < 0.2 + 3 * np.sqrt(0.2 * 0.8 / (225 * G))
    armies = np.array(armies)
    assert armies.min() == 40 and armies.max() == 50
    hist = np.bincount(armies - 40, minlength=11)
    exp = len(armies) / 11
    assert float(((hist - exp) ** 2 / exp).sum()) < 29.6  # 99.9% of chi2(10)


def test_generator_mountain_extremes():
    env = make_env(20, 9, 9, auto_reset=0, mountain_thresh=0, n_cities=0)
    for g in range(20):
        assert not np.any(env.board(g)[2] == T_MTN)
    env = make_env(20, 9, 9, auto_reset=0, mountain_thresh=0xFFFFFFFF, n_cities=3)
    for g in range(20):
        a, o, t = env.board(g)
        gens = np.flatnonzero(t == T_GEN)
        assert len(gens) == 2
        lab, _ = ndimage.label((t != T_MTN).reshape(9, 9))
        assert lab.reshape(-1)[gens[0]] == lab.reshape(-1)[gens[1]]


@pytest.mark.parametrize("mode,P,H,W", [(1, 4, 20, 20), (2, 8, 20, 22), (2, 8, 3, 3), (0, 2, 1, 2)])
def test_generator_places_all_generals(mode, P, H, W):
    env = make_env(30, H, W, mode, P, auto_reset=0, n_cities=-1, city_per_mille=30)
    for g in range(30):
        a, o, t = env.board(g)
        gens = np.flatnonzero(t == T_GEN)
        assert len(gens) == P
        assert sorted(o[gens].tolist()) == list(range(P))
        lab, _ = ndimage.label((t != T_MTN).reshape(H, W))
        assert len(set(lab.reshape(-1)[gens].tolist())) == 1
        assert (t == T_CASTLE).sum() <= (H * W * 30) // 1000


def test_generator_depends_on_game_and_epoch():
    env = make_env(4, 10, 10, auto_reset=0)
    boards = [env.board(g)[2].copy() for g in range(4)]
    assert all(not np.array_equal(boards[0], b) for b in boards[1:])
    env2 = make_env(4, 10, 10, auto_reset=0)
    for g in range(4):
        np.testing.assert_array_equal(env2.board(g)[2], boards[g])
    env2.reset([1])
    assert env2.scalars(1)["epoch"] == 1
    assert not np.array_equal(env2.board(1)[2], boards[1])
    env3 = make_env(4, 10, 10, auto_reset=0, game_id_base=1)  # local game 0 is global game 1
    np.testing.assert_array_equal(env3.board(0)[2], boards[1])


# ---------------------------------------------------------------- policy
def test_policy_uniform_and_legal():
    rng = np.random.default_rng(8)
    H, W = 5, 6
    env = make_env(1, H, W, 0, 2, auto_reset=0)
    army, owner, terrain = _random_state(rng, H, W, 2, 0)
    env.set_game(0, army, owner, terrain)
    mask = env.observe(0, 0)["mask"]
    legal = [(c, d) for c in range(H * W) for d in range(4) if (mask[c] >> d) & 1]
    assert len(legal) >= 4
    counts = {x: 0 for x in legal}
    splits = 0
    n = 6000
    for f in range(n):
        env.set_game(0, army, owner, terrain, frame=f)
        a = int(env.policy(policy_seed=2)[0, 0])
        c, k = divmod(a, 9)
        assert 1 <= k <= 8
        d = (k - 1) % 4
        counts[(c, d)] += 1
        splits += k >= 5
    exp = n / len(legal)
    chi2 = sum((v - exp) ** 2 / exp for v in counts.values())
    dof = len(legal) - 1
    assert chi2 < dof + 5 * np.sqrt(2 * dof)
    assert abs(splits / n - SPLIT / 2**32) < 4 * np.sqrt(0.2 * 0.8 / n)


def test_policy_passes_without_legal_moves():
    env = make_env(1, 1, 3, 0, 2, auto_reset=0)
    env.set_game(0, np.array([1, 0, 1], np.int16), np.array([0, -1, 1], np.int8), np.array([3, 0, 3], np.int8))
    assert env.policy(5)[0, :2].tolist() == [0, 0]


# ---------------------------------------------------------------- invariants
def check_invariants(env, g, prev_total, prev_alive):
    a, o, t = env.board(g)
    s = env.scalars(g)
    P = int(env.P[g])
    assert np.all(o >= -1) and np.all(o < P)
    assert np.all(a >= 0)
    assert np.all(o[t == T_MTN] == -1) and np.all(a[t == T_MTN] == 0)
    gens = np.flatnonzero(t == T_GEN)
    for p in range(P):
        if (s["alive"] >> p) & 1:
            assert np.sum(o[gens] == p) == 1, "alive player holds exactly one general"
        else:
            assert not np.any(o == p), "eliminated player owns nothing"
    if prev_total is not None and s["epoch"] == prev_alive[1] and s["alive"] == prev_alive[0] and not s["done"]:
        turn = s["turn"]
        owned = o >= 0
        growth = 0
        if turn % 2 == 0:
            growth += int(np.sum(owned & ((t == T_GEN) | (t == T_CASTLE))))
        if turn % 50 == 0:
            growth += int(np.sum(owned & (t == T_PLAIN)))
        delta = int(a.astype(np.int64).sum()) - prev_total
        if s["saturated"] == 0:
            lost = growth - delta
            assert lost >= 0 and lost % 2 == 0, (delta, growth)
    return int(a.astype(np.int64).sum()), (s["alive"], s["epoch"])


@pytest.mark.parametrize("mode,P,H,W", [(0, 2, 8, 8), (1, 4, 8, 9), (2, 6, 9, 9)])
def test_invariants_random_rollout(mode, P, H, W):
    G = 6
    env = make_env(G, H, W, mode, P, seed=3, min_general_dist=2, n_cities=2, max_turns=150)
    prev = [(None, None)] * G
    ends = 0
    for f in range(400):
        acts = env.policy(policy_seed=9)
        env.step(acts)
        for g in range(G):
            ends += env.scalars(g)["done"] != 0
            prev[g] = check_invariants(env, g, *prev[g]) if prev[g][0] is not None else check_invariants(
                env, g, None, None)
            assert env.scalars(g)["frame"] == f + 1
    assert ends > 0


def test_exhaustive_joint_actions_3x3():
    """All 81 x 81 joint actions on hand-built 3x3 1v1 positions."""
    positions = [
        ("6@0G 3@0 0", "M 4@1 2@1", "0 0 5@1G"),
        ("5@0G 45C 0", "3@0 M 9@1", "2@1 0 4@1G"),
        ("2@0G 7@1 3@1G", "2@0 1@1 0", "0 0 M"),
    ]
    import golden_io
    env = make_env(1, 3, 3, 0, 2, auto_reset=0)
    for rows in positions:
        army, owner, terrain = golden_io.parse_board(list(rows), 3, 3)
        total0 = int(army.astype(np.int64).sum())
        for turn in (0, 1):
            for a0, a1 in itertools.product(range(81), range(81)):
                env.set_game(0, army, owner, terrain, turn=turn)
                env.step(np.array([[a0, a1]], np.int32))
                a, o, t = env.board(0)
                s = env.scalars(0)
                assert np.all(o >= -1) and np.all(o < 2) and np.all(a >= 0)
                assert np.all(o[t == T_MTN] == -1) and np.all(a[t == T_MTN] == 0)
                alive = s["alive"]
                for p in range(2):
                    if (alive >> p) & 1:
                        assert np.sum((t == T_GEN) & (o == p)) == 1
                    else:
                        assert not np.any(o == p)
                growth = int(np.sum((o >= 0) & ((t == T_GEN) | (t == T_CASTLE)))) if s["turn"] % 2 == 0 else 0
                lost = total0 + growth - int(a.astype(np.int64).sum())
                if alive == 3:
                    assert lost >= 0 and lost % 2 == 0
                    assert s["done"] == 0
                else:
                    assert s["done"] == 1 and bin(alive).count("1") == 1
                    w = 0 if alive == 1 else 1
                    assert s["reward"][w] == 1.0 and s["reward"][1 - w] == -1.0


def test_auto_reset_matches_generator():
    """After a finished game the board is the generator's map of the next epoch."""
    G = 8
    env = make_env(G, 4, 4, 0, 2, seed=21, min_general_dist=1, n_cities=1)
    fresh = make_env(G, 4, 4, 0, 2, seed=21, min_general_dist=1, n_cities=1, auto_reset=0)
    seen = 0
    for f in range(300):
        env.step(env.policy(policy_seed=4))
        for g in range(G):
            s = env.scalars(g)
            if s["done"]:
                seen += 1
                fresh.reset([g])
                assert fresh.scalars(g)["epoch"] == s["epoch"]
                for x, y in zip(env.board(g), fresh.board(g)):
                    np.testing.assert_array_equal(x, y)
                assert s["turn"] == 0 and s["alive"] == 3
    assert seen >= 5


def test_truncation_and_frozen_games():
    env = make_env(2, 6, 6, 0, 2, max_turns=5, auto_reset=0)
    for t in range(5):
        env.step(np.zeros((2, 2), np.int32))
    s = env.scalars(0)
    assert s["done"] == 2 and s["finished"] == 1 and list(s["reward"][:2]) == [0, 0]
    board = [x.copy() for x in env.board(0)]
    env.step(np.zeros((2, 2), np.int32))
    s = env.scalars(0)
    assert s["done"] == 0 and s["frame"] == 6 and s["turn"] == 5
    for x, y in zip(env.board(0), board):
        np.testing.assert_array_equal(x, y)
    assert not np.any(env.observe(0, 0)["mask"])


def test_workload_shapes_are_seeded():
    a = shapes(100, (15, 30), seed=4)
    b = shapes(100, (15, 30), seed=4)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    H, W, mode, P = shapes(1000, (20, 40), ((0, 0.4), (1, 0.3), (2, 0.3)), seed=1)
    assert H.min() >= 20 and H.max() <= 40
    assert abs(np.mean(mode == 1) - 0.3) < 0.01 and set(np.unique(P)) == {2, 4, 8}


def test_two_player_free_for_all_is_1v1():
    """With two players a free-for-all game follows exactly the 1v1 rules
    (Sec. III: teams exist only in 2v2; elimination ends a game of two either
    way), so the two modes give the same maps, moves, outputs and rewards
    frame by frame.  The GPU runs both through the same two-player kernels."""
    G = 24
    rng = np.random.default_rng(3)
    H = rng.integers(4, 16, G).astype(np.int32)
    W = rng.integers(4, 16, G).astype(np.int32)
    kw = dict(seed=5, min_general_dist=1, n_cities=3, max_turns=60)
    a = OracleEnv(H, W, np.zeros(G, np.int32), np.full(G, 2, np.int32), **kw)
    b = OracleEnv(H, W, np.full(G, 2, np.int32), np.full(G, 2, np.int32), **kw)
    resets = 0
    for f in range(200):
        act = a.policy(4)
        assert np.array_equal(act, b.policy(4)), f"policy differs at frame {f}"
        a.step(act)
        b.step(act)
        for g in range(G):
            for x, y in zip(a.board(g), b.board(g)):
                assert np.array_equal(x, y), f"board of game {g} differs at frame {f}"
            sa, sb = a.scalars(g), b.scalars(g)
            assert sa["reward"].tolist() == sb["reward"].tolist() and sa["done"] == sb["done"]
            resets += sa["done"] != 0
            for p in range(2):
                oa, ob = a.observe(g, p), b.observe(g, p)
                for k in oa:
                    assert np.array_equal(oa[k], ob[k]), f"{k} of game {g} player {p} differs at frame {f}"
    assert resets > 0, "expected finished games"
