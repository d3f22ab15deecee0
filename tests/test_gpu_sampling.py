"""Policy sampling over the H x W x 9 action space and the expanded legal
mask on the GPU vs the oracle, through the C-ABI.  Both sides draw with an
exact integer inverse CDF over a bit-reproducible exponential, so actions
and masks must agree exactly."""
import numpy as np
import pytest

from gpu_helpers import compare_frame, flat_to_rows
from oracle import OracleEnv
from paper_2606_23348_gb300.workloads import shapes, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_23348_gb300.build import build_library
    build_library()


def oracle_logits(env, flat, games=None):
    """Per game [P][N * 9] slices of the library's logits layout."""
    games = range(env.G) if games is None else games
    res = []
    for g in games:
        npad, N, P = int(env.npad[g]), int(env.N[g]), int(env.P[g])
        rows = []
        for p in range(P):
            q = int(env.plane_off[g]) + p * npad
            rows.append(flat[q * 9:q * 9 + 9 * N])
        res.append(np.stack(rows))
    return res


def check_sample(env, orc, logits, seed, tag, games=None):
    import torch
    acts = env.new_actions()
    mask9 = torch.full((int(env.layout.plane_cells) * 9,), 7, dtype=torch.uint8, device="cuda")
    env.sample_actions(logits, seed, acts, mask9)
    torch.cuda.synchronize()
    flat = logits.cpu().numpy()
    want_a, want_m = orc.sample_actions(oracle_logits(env, flat, games), seed)
    got_a = flat_to_rows(env, acts.cpu().numpy())
    m9 = mask9.cpu().numpy()
    games = range(env.G) if games is None else games
    for k, g in enumerate(games):
        P, N, npad = int(env.P[g]), int(env.N[g]), int(env.npad[g])
        np.testing.assert_array_equal(got_a[g, :P], want_a[k, :P], err_msg=f"{tag} game {g}: actions")
        for p in range(P):
            q = int(env.plane_off[g]) + p * npad
            np.testing.assert_array_equal(m9[q * 9:q * 9 + 9 * N], want_m[k][p], err_msg=f"{tag} game {g} p {p}")
            assert not m9[q * 9 + 9 * N:(q + npad) * 9].any(), f"{tag} game {g}: padding entries"
    return acts


def pair(H, W, mode, P, **kw):
    from paper_2606_23348_gb300.generals import GeneralsEnv
    return GeneralsEnv(H, W, mode, P, **kw), OracleEnv(H, W, mode, P, **kw)


# the spreads of a game over the GPU: one warp per game, one CTA per game,
# one CTA per player with a thread per (own cell, entry)
FORMS = pytest.mark.parametrize("form", [1, 2, 3], ids=["warp", "cta", "wide"])


@FORMS
@pytest.mark.parametrize("scale", [0.0, 3.0, 40.0])
def test_sampling_matches_oracle_mixed_modes(scale, form):
    import torch
    G = 30
    H, W, mode, P = shapes(G, (3, 14), ((0, 0.4), (1, 0.3), (2, 0.3)), seed=5)
    env, orc = pair(H, W, mode, P, seed=8, n_cities=2)
    env.set_sample_form(form)
    acts = env.new_actions()
    out = env.new_outputs()
    env.policy(3, acts)
    for f in range(15):
        a = orc.policy(3)
        env.step_policy(acts, out, 3, acts)
        orc.step(a)
    gen = torch.Generator(device="cuda").manual_seed(11)
    for s in range(4):
        logits = torch.randn(int(env.layout.plane_cells) * 9, generator=gen, device="cuda") * scale
        check_sample(env, orc, logits, 100 + s, f"scale {scale} seed {s}")


def test_device_rollout_from_logits():
    """Self-play shape: logits -> sampled actions -> step, all on the device; the
    oracle replays the same logits; every state and output compared."""
    import torch
    G = 20
    H, W, mode, P = shapes(G, (5, 12), ((0, 0.5), (2, 0.5)), seed=6)
    env, orc = pair(H, W, mode, P, seed=4, n_cities=2, max_turns=30)
    out = env.new_outputs()
    gen = torch.Generator(device="cuda").manual_seed(2)
    for f in range(60):
        logits = torch.randn(int(env.layout.plane_cells) * 9, generator=gen, device="cuda") * 2.0
        acts = check_sample(env, orc, logits, 7, f"frame {f}")
        a_orc, _ = orc.sample_actions(oracle_logits(env, logits.cpu().numpy()), 7)
        env.step(acts, out)
        orc.step(a_orc)
        compare_frame(env, out, orc, f"frame {f}")


@FORMS
@pytest.mark.parametrize("H,W,mode,P", [(1, 2, 0, 2), (40, 1, 2, 3), (64, 64, 2, 8), (3, 3, 2, 8)])
def test_sampling_edge_shapes(H, W, mode, P, form):
    import torch
    env, orc = pair([H, H], [W, W], [mode, mode], [P, P], seed=5, n_cities=1)
    env.set_sample_form(form)
    acts = env.new_actions()
    out = env.new_outputs()
    env.policy(1, acts)
    for f in range(6):
        a = orc.policy(1)
        env.step_policy(acts, out, 1, acts)
        orc.step(a)
    logits = torch.randn(int(env.layout.plane_cells) * 9, device="cuda")
    check_sample(env, orc, logits, 9, f"edge {H}x{W}")


@FORMS
def test_sampling_large_territories(form):
    """Planted boards where one player owns most of a large board (hundreds of
    own cells, thousands of legal entries: several rounds of every form's
    passes, beyond what any form keeps in registers) and the others hold a
    few cells each; 1v1, 2v2 and FFA-8, armies 0..30, some cells with a
    single unit (only the pass entry legal)."""
    import torch
    shp = [(32, 32, 0, 2), (40, 37, 1, 4), (20, 24, 2, 8), (64, 64, 0, 2)]
    H, W, mode, P = (np.array([x[i] for x in shp], np.int32) for i in range(4))
    env, orc = pair(H, W, mode, P, seed=2, n_cities=0)
    env.set_sample_form(form)
    rng = np.random.default_rng(17)
    n = int(env.layout.state_cells)
    army, owner, terrain = np.zeros(n, np.int16), np.full(n, -1, np.int8), np.zeros(n, np.int8)
    sc = np.zeros((env.G, 8), np.uint32)
    for g in range(env.G):
        N, Pg, o = int(env.N[g]), int(P[g]), int(env.state_off[g])
        t = np.where(rng.random(N) < 0.08, 1, 0).astype(np.int8)  # mountains
        ow = np.where(rng.random(N) < 0.75, 0, rng.integers(-1, Pg, N)).astype(np.int8)
        ow[t == 1] = -1
        a = np.where(ow >= 0, rng.integers(0, 31, N), 0).astype(np.int16)
        a[(ow >= 0) & (rng.random(N) < 0.2)] = 1
        free = np.flatnonzero(t == 0)
        for q, c in enumerate(rng.choice(free, Pg, replace=False)):  # one general per player
            ow[c], t[c], a[c] = q, 3, 5
        army[o:o + N], owner[o:o + N], terrain[o:o + N] = a, ow, t
        sc[g, 0], sc[g, 1], sc[g, 3] = 60, 4, (1 << Pg) - 1
        orc.set_game(g, a, ow, t, turn=60, frame=4)
    env.write_state(army, owner, terrain, sc)
    gen = torch.Generator(device="cuda").manual_seed(5)
    for s in range(3):
        logits = torch.randn(int(env.layout.plane_cells) * 9, generator=gen, device="cuda") * (1.0 + 4 * s)
        check_sample(env, orc, logits, 40 + s, f"territories seed {s}")


def test_expand_mask_only_and_errors():
    import torch
    from paper_2606_23348_gb300.generals import GeneralsError
    env, orc = pair([6, 7], [6, 9], [0, 2], [2, 3], seed=1)
    m9 = env.expand_mask()
    torch.cuda.synchronize()
    logits = env.new_logits()
    m9b = torch.empty_like(m9)
    env.sample_actions(logits, 1, None, m9b)
    torch.cuda.synchronize()
    assert torch.equal(m9, m9b)
    for form in (1, 2, 3):  # the mask of every spread, and the actions with it
        env.set_sample_form(form)
        m9c, a1 = torch.empty_like(m9), env.sample_actions(logits, 1)
        a2 = env.sample_actions(logits, 1, None, m9c)
        torch.cuda.synchronize()
        assert torch.equal(m9, m9c) and torch.equal(a1, a2)
    for form in (-1, 4):
        with pytest.raises(GeneralsError):
            env.set_sample_form(form)
    assert env.lib.gen_sample_actions(env.h, None, 0, None, None, None) != 0  # nothing to compute
    with pytest.raises(GeneralsError):
        env.sample_actions(logits[1:], 1)  # misaligned logits
    m9x = torch.empty(int(env.layout.plane_cells) * 9 + 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(GeneralsError):
        env.sample_actions(logits, 1, None, m9x[4:])  # a mask 4 but not 16 bytes aligned: refused on the host


def test_sampling_full_size_24x24_65536_sampled():
    """The 65,536-game workload: every player sampled on the GPU; three blocks of
    32 games replayed by the oracle."""
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv
    H, W, mode, P, gen, _ = workload("1v1-65536x24x24")
    env = GeneralsEnv(H, W, mode, P, seed=1, **gen)
    acts = env.new_actions()
    out = env.new_outputs()
    env.policy(2, acts)
    for f in range(5):
        env.step_policy(acts, out, 2, acts)
    g = torch.Generator(device="cuda").manual_seed(5)
    logits = torch.randn(int(env.layout.plane_cells) * 9, generator=g, device="cuda") * 2.0
    got = env.sample_actions(logits, 77)
    torch.cuda.synchronize()
    flat = logits.cpu().numpy()
    ga = got.cpu().numpy()
    for start in (0, 30000, 65536 - 32):
        n = 32
        orc = OracleEnv(H[start:start + n], W[start:start + n], mode[start:start + n], P[start:start + n], seed=1,
                        game_id_base=start, **gen)
        for f in range(5):
            orc.step(orc.policy(2))
        want, _ = orc.sample_actions(oracle_logits(env, flat, range(start, start + n)), 77)
        np.testing.assert_array_equal(ga[2 * start:2 * (start + n)], want[:, :2].reshape(-1))


def test_selfplay_loop_in_a_cuda_graph_matches_plain_launches():
    """Sample -> step -> features, 8 frames captured as one CUDA graph and
    replayed, gives the same actions, state and features as plain launches."""
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv
    outs = []
    for use_graph in (False, True):
        env = GeneralsEnv(11, 13, 0, 2, batch=96, seed=6, n_cities=3, max_turns=9)
        fb = env.features(3, 8)
        out, acts = env.new_outputs(), env.new_actions()
        x, tok = fb.new_output(), fb.new_series()
        logits = torch.randn(int(env.layout.plane_cells) * 9, generator=torch.Generator(device="cuda").manual_seed(3),
                             device="cuda")
        s = torch.cuda.Stream()

        def frame():
            env.sample_actions(logits, 5, acts)
            env.step(acts, out)
            fb.build(x, tok)

        with torch.cuda.stream(s):
            frame()  # first calls outside any capture
        torch.cuda.synchronize()
        if use_graph:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s):
                for _ in range(8):
                    frame()
            graph.replay()
        else:
            with torch.cuda.stream(s):
                for _ in range(8):
                    frame()
        torch.cuda.synchronize()
        st = env.read_state()
        outs.append((acts.cpu(), x.cpu(), tok.cpu(), [torch.from_numpy(a.copy()) for a in st]))
    (a0, x0, t0, s0), (a1, x1, t1, s1) = outs
    assert torch.equal(a0, a1) and torch.equal(x0, x1) and torch.equal(t0, t1)
    assert all(torch.equal(u, v) for u, v in zip(s0, s1))
