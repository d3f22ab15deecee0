"""Feature tensor (App. A) on the GPU vs the oracle, through the C-ABI.

Every channel of every player and game is compared element by element with
the oracle's builder run on the same frames: exact for every channel except
the age row (log(1 + dt) / 5), where both sides evaluate the logarithm in
double precision and round once to float, so they may differ by at most one
float ulp when the two libraries' double logarithms differ in their last
bit.  Padding cells must read 0 in every channel.
"""
import os

import numpy as np
import pytest

from oracle import OracleEnv
from oracle.orc import OracleFeatures
from paper_2606_23348_gb300.workloads import shapes, workload

pytestmark = pytest.mark.gpu

AGE = 21


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_23348_gb300.build import build_library
    build_library()


def compare_series(env, fb, series, want, tag, games=None):
    """Temporal tokens: exact int32 equality per player slot."""
    import torch
    torch.cuda.synchronize()
    got = series.cpu().numpy()
    games = range(env.G) if games is None else games
    T = fb.window
    for k, g in enumerate(games):
        for p in range(int(env.P[g])):
            s = int(env.player_off[g]) + p
            np.testing.assert_array_equal(got[s * 2 * T:(s + 1) * 2 * T].reshape(T, 2), want[k][p],
                                          err_msg=f"{tag} game {g} player {p}: temporal tokens")


def compare_features(env, fb, out, want, tag, games=None, orc_index=None):
    import torch
    torch.cuda.synchronize()
    C = fb.channels
    games = range(env.G) if games is None else games
    for k, g in enumerate(games):
        npad, N, P = int(env.npad[g]), int(env.N[g]), int(env.P[g])
        for p in range(P):
            q = int(env.plane_off[g]) + p * npad
            got = out[q * C:q * C + C * npad].view(C, npad).cpu().numpy()
            w = want[k if orc_index is None else orc_index(k)][p]
            assert not got[:, N:].any(), f"{tag} game {g} player {p}: padding cells not zero"
            exact = np.ones(C, bool)
            exact[AGE] = False
            if not np.array_equal(got[exact, :N], w[exact]):
                bad = np.argwhere(got[:, :N] != w)
                ch, c = bad[0]
                raise AssertionError(f"{tag} game {g} player {p}: channel {ch} cell {c}: gpu {got[ch, c]} oracle "
                                     f"{w[ch, c]} ({len(bad)} differences)")
            np.testing.assert_array_max_ulp(got[AGE, :N], w[AGE], maxulp=1)


def lockstep(env, orc, fb, ofb, frames, policy_seed, tag, every=1, subset_reset=None):
    import torch
    out = env.new_outputs()
    acts = env.new_actions()
    fout = fb.new_output()
    ser = fb.new_series() if fb.window else None
    env.observe(out)
    fb.build(fout, ser)
    compare_features(env, fb, fout, ofb.build(), f"{tag} create")
    if ser is not None:
        compare_series(env, fb, ser, ofb.series, f"{tag} create")
    env.policy(policy_seed, acts)
    for f in range(frames):
        a = orc.policy(policy_seed)
        env.step_policy(acts, out, policy_seed, acts)
        orc.step(a)
        if subset_reset is not None and f == frames // 2:
            ids = np.asarray(subset_reset, np.int32)
            env.reset(out, torch.from_numpy(ids).cuda())
            orc.reset(ids)
            env.policy(policy_seed, acts)  # the reset games' actions come from their new maps
        fb.build(fout, ser)
        want = ofb.build()
        if (f + 1) % every == 0 or f == frames - 1:
            compare_features(env, fb, fout, want, f"{tag} frame {f + 1}")
            if ser is not None:
                compare_series(env, fb, ser, ofb.series, f"{tag} frame {f + 1}")
    return fout


def pair(H, W, mode, P, hist=7, window=0, form=0, **kw):
    from paper_2606_23348_gb300.generals import GeneralsEnv
    env = GeneralsEnv(H, W, mode, P, **kw)
    orc = OracleEnv(H, W, mode, P, **kw)
    fb = env.features(hist, window)
    if form:
        fb.set_form(form)
    return env, orc, fb, OracleFeatures(orc, hist, window)


# both spreads of a game over the GPU: one warp per game, one CTA per game
FORMS = pytest.mark.parametrize("form", [1, 2], ids=["warp", "cta"])


@FORMS
def test_features_mixed_modes_with_resets(form):
    """Ragged 1v1 / 2v2 / FFA boards, truncation resets every 25 turns, every frame compared."""
    G = 24
    H, W, mode, P = shapes(G, (4, 12), ((0, 0.4), (1, 0.3), (2, 0.3)), seed=8)
    env, orc, fb, ofb = pair(H, W, mode, P, window=32, form=form, seed=4, n_cities=2, max_turns=25)
    lockstep(env, orc, fb, ofb, 80, 6, "mixed")


@FORMS
@pytest.mark.parametrize("hist,window", [(1, 512), (16, 1)])
def test_features_history_lengths(hist, window, form):
    H, W, mode, P, gen, _ = workload("1v1-64x15x15")
    env, orc, fb, ofb = pair(H[:16], W[:16], mode[:16], P[:16], hist=hist, window=window, form=form, seed=1, **gen)
    assert fb.channels == 24 + 2 * hist
    lockstep(env, orc, fb, ofb, 30, 3, f"hist {hist}", every=3)


@FORMS
@pytest.mark.parametrize("hist", [7, 16])
def test_features_large_boards_and_odd_player_counts(form, hist):
    """64x64 FFA-8 (256 (player, 128-cell) items: several batches per warp in
    the CTA form, the most staging shared memory allows at hist 16), FFA-3 on
    40x37 and 3x5 (an odd player count: unaligned bitset regions), and a 1x2
    board, with truncation resets; every frame compared."""
    H, W, mode, P = (np.array(v, np.int32) for v in ([64, 40, 3, 1], [64, 37, 5, 2], [2, 2, 2, 0], [8, 3, 3, 2]))
    env, orc, fb, ofb = pair(H, W, mode, P, hist=hist, window=16, form=form, seed=6, n_cities=3, max_turns=12)
    lockstep(env, orc, fb, ofb, 30, 5, f"large hist {hist}", every=2)


@FORMS
def test_features_subset_reset_and_repeat_build(form):
    """A reset of some games clears their memory; a second build in one frame changes nothing."""
    G = 12
    H, W, mode, P = shapes(G, (6, 9), ((0, 0.5), (2, 0.5)), seed=2)
    env, orc, fb, ofb = pair(H, W, mode, P, window=7, form=form, seed=3, n_cities=2)
    fout = lockstep(env, orc, fb, ofb, 20, 5, "subset", subset_reset=[0, 5, 11])
    again = fb.build()
    import torch
    torch.cuda.synchronize()
    assert torch.equal(fout, again)


@FORMS
@pytest.mark.parametrize("H,W,mode,P", [(1, 2, 0, 2), (40, 1, 2, 3), (33, 5, 1, 4), (64, 64, 2, 8), (3, 3, 2, 8)])
def test_features_edge_shapes(H, W, mode, P, form):
    env, orc, fb, ofb = pair([H, H], [W, W], [mode, mode], [P, P], window=3, form=form, seed=5, n_cities=1,
                             max_turns=15)
    lockstep(env, orc, fb, ofb, 20, 9, f"edge {H}x{W}", every=4)


def _golden_cases():
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "features")
    return sorted(os.path.join(d, f) for f in os.listdir(d) if f.endswith(".txt") and f != "README.txt")


@pytest.mark.parametrize("path", _golden_cases(), ids=lambda p: os.path.basename(p)[:-4])
def test_feature_golden_on_gpu(path):
    """The hand-worked feature scenarios, loaded into the GPU state."""
    import torch
    from test_oracle_features import load_feature_case
    from paper_2606_23348_gb300.generals import GeneralsEnv
    sc = load_feature_case(path)
    P = sc["P"]
    env = GeneralsEnv([sc["H"]], [sc["W"]], [sc["mode"]], [P], seed=7, auto_reset=0, n_cities=0,
                      min_general_dist=1)
    army, owner, terrain = sc["board"]
    npad = int(env.npad[0])
    pad = lambda x, v: np.concatenate([x, np.full(npad - x.shape[0], v, x.dtype)])
    scal = np.array([[sc["turn"], 0, 0, (1 << P) - 1, 0, 0, 0, 0]], np.uint32)
    env.write_state(pad(army, 0), pad(owner, -1), pad(terrain, 0), scal)
    fb = env.features(sc["hist"], sc.get("window", 0))
    out = env.new_outputs()
    ser = fb.new_series() if fb.window else None
    n = 0
    for fr in sc["frames"]:
        if fr["actions"] is not None:
            env.step(torch.from_numpy(fr["actions"][:P].copy()).cuda(), out)
        f = fb.build(series=ser)
        torch.cuda.synchronize()
        for p, k, army, land in fr["series"]:
            assert tuple(fb.player_series(ser, 0, p)[k].tolist()) == (army, land)
            n += 1
        for p, ch, want in fr["checks"]:
            got = fb.player_view(f, 0, p)[ch].cpu().numpy().astype(np.float64)
            np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-9, err_msg=f"player {p} channel {ch}")
            n += 1
    assert n > 10


@FORMS
def test_features_full_size_24x24_65536_sampled(form):
    """65,536 games of 24x24: features built every frame on the GPU; three
    blocks of 32 games replayed by the oracle and compared at the end."""
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv
    H, W, mode, P, gen, _ = workload("1v1-65536x24x24")
    env = GeneralsEnv(H, W, mode, P, seed=1, **gen)
    fb = env.features(7, 512)
    fb.set_form(form)
    out = env.new_outputs()
    acts = env.new_actions()
    fout = fb.new_output()
    ser = fb.new_series()
    env.policy(2, acts)
    fb.build(fout, ser)
    frames = 12
    for f in range(frames):
        env.step_policy(acts, out, 2, acts)
        fb.build(fout, ser)
    torch.cuda.synchronize()
    for start in (0, 40000, 65536 - 32):
        n = 32
        orc = OracleEnv(H[start:start + n], W[start:start + n], mode[start:start + n], P[start:start + n], seed=1,
                        game_id_base=start, **gen)
        ofb = OracleFeatures(orc, 7, 512)
        ofb.build()
        for f in range(frames):
            orc.step(orc.policy(2))
            want = ofb.build()
        compare_features(env, fb, fout, want, f"full size block {start}", games=range(start, start + n))
        compare_series(env, fb, ser, ofb.series, f"full size block {start}", games=range(start, start + n))


def test_feature_builder_argument_errors():
    """Bad arguments are refused with an error code and a message, not a fault."""
    import ctypes as C
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv, GeneralsError
    env = GeneralsEnv(6, 7, 0, 2, batch=3, seed=1)
    lib = env.lib
    h = C.c_void_p()
    for hist, window in ((0, 0), (17, 0), (7, -1), (7, 4097)):
        assert lib.gen_features_create_ex(C.byref(h), env.h, hist, window) != 0
        assert lib.gen_last_error()
    fb = env.features(3)
    out = fb.new_output()
    with pytest.raises(GeneralsError):
        fb.build(out, torch.zeros(16, dtype=torch.int32, device="cuda"))  # no temporal window
    assert lib.gen_features_build(fb.h, C.c_void_p(out.data_ptr() + 4), None) != 0  # misaligned
    assert lib.gen_features_build(fb.h, None, None) != 0
    for form in (-1, 3):
        with pytest.raises(GeneralsError):
            fb.set_form(form)
    fb.build(out)  # still usable
    torch.cuda.synchronize()


def test_age_row_every_dt_up_to_65535_bit_exact():
    """The age row log(1 + dt) / 5 (App. A row 21, Q31) for every dt in
    [0, 65535], bit for bit against the oracle: the library evaluates the
    logarithm with CUDA's double log and the oracle with the host C library's,
    each rounding once to float.  One game per dt on a 1 x 6 board: at turn
    100 player 1 holds the cell next to player 0's general (seen), then the
    generals swap ends and the turn moves on by dt, so player 0 remembers an
    enemy in fog there for dt turns."""
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv
    G, N = 65536, 6
    kw = dict(seed=1, n_cities=0, min_general_dist=1)
    env = GeneralsEnv(1, N, 0, 2, batch=G, **kw)
    orc = OracleEnv(np.ones(G, np.int32), np.full(G, N, np.int32), np.zeros(G, np.int32), np.full(G, 2, np.int32), **kw)
    fb, ofb = env.features(7), OracleFeatures(orc, 7)
    npad = int(env.npad[0])

    def place(terrain, owner, army, turns, frame):
        a = np.zeros((G, npad), np.int16)
        o = np.full((G, npad), -1, np.int8)
        t = np.zeros((G, npad), np.int8)
        a[:, :N], o[:, :N], t[:, :N] = army, owner, terrain
        sc = np.zeros((G, 8), np.uint32)
        sc[:, 0], sc[:, 1], sc[:, 3] = turns, frame, 3
        env.write_state(a.reshape(-1), o.reshape(-1), t.reshape(-1), sc)
        for g in range(G):
            orc.set_game(g, army, owner, terrain, turn=int(turns[g]), frame=frame)

    # seen: player 1's plain next to player 0's general
    place([3, 0, 0, 0, 0, 3], [0, 1, -1, -1, -1, 1], [5, 3, 0, 0, 0, 5], np.full(G, 100), 1)
    out = fb.build()
    compare_features(env, fb, out, ofb.build(), "seen", games=range(0, G, 4099), orc_index=lambda k: 4099 * k)
    # fogged for dt = g turns: the generals swap ends, the cell is neutral again
    dts = np.arange(G, dtype=np.int64)
    place([3, 0, 0, 0, 0, 3], [1, -1, -1, -1, -1, 0], [5, 0, 0, 0, 0, 5], 100 + dts, 2)
    out = fb.build()
    want = ofb.build()
    torch.cuda.synchronize()
    C = fb.channels
    got = out.view(G, 2, C, npad)[:, 0, AGE, 1].cpu().numpy()
    exp = np.array([w[0][AGE][1] for w in want], np.float32)
    assert exp[0] == 0.0 and exp[1] > 0.0  # dt = 0 gives log(1) = 0; the row is live
    bad = np.flatnonzero(got.view(np.uint32) != exp.view(np.uint32))
    assert bad.size == 0, f"age row differs at dt {bad[:10].tolist()} ({bad.size} values)"
    # and every channel of a spread of games, against the oracle
    compare_features(env, fb, out, [want[g] for g in range(0, G, 997)], "fogged", games=range(0, G, 997))
