"""CUDA path vs the oracle, bit-exact on every state and output byte.

All tests call the library through its C-ABI (ctypes binding) on cuda:0.
"""
import numpy as np
import pytest

import golden_io
from gpu_helpers import compare_frame, flat_to_rows, oracle_actions_flat
from oracle import OracleEnv
from paper_2606_23348_gb300.workloads import random_actions, shapes, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_23348_gb300.build import build_library
    build_library()


def pair(H, W, mode, n_players, lanes=0, **kw):
    from paper_2606_23348_gb300.generals import GeneralsEnv
    env = GeneralsEnv(H, W, mode, n_players, **kw)
    if lanes:
        env.set_lane_groups(lanes)
    orc = OracleEnv(H, W, mode, n_players, **kw)
    return env, orc


# games per warp in the step kernels: one, by batch size, or two (four in
# rollouts) wherever the games allow
LANES = pytest.mark.parametrize("lanes", [1, 2], ids=["warp", "narrow"])
LANES_AUTO = pytest.mark.parametrize("lanes", [0, 2], ids=["auto", "narrow"])


def rollout_policy(env, orc, frames, policy_seed=2, check_every=1, tag=""):
    out = env.new_outputs()
    acts = env.new_actions()
    env.observe(out)
    compare_frame(env, out, orc, f"{tag} create")
    env.policy(policy_seed, acts)
    for f in range(frames):
        a_orc = orc.policy(policy_seed)
        got = acts.cpu().numpy()
        want = oracle_actions_flat(env, a_orc)
        if not np.array_equal(got, want):
            i = int(np.flatnonzero(got != want)[0])
            raise AssertionError(f"{tag} frame {f}: policy slot {i} gpu {got[i]} oracle {want[i]}")
        env.step_policy(acts, out, policy_seed, acts)
        orc.step(a_orc)
        if (f + 1) % check_every == 0 or f == frames - 1:
            compare_frame(env, out, orc, f"{tag} frame {f + 1}")
    return out


@LANES
def test_c0_1v1_64x15x15_500_turns(lanes):
    """The 64-game 15x15 1v1 workload, 500 turns of the benchmark policy, every frame compared."""
    H, W, mode, P, gen, frames = workload("1v1-64x15x15")
    env, orc = pair(H, W, mode, P, lanes=lanes, seed=1, **gen)
    rollout_policy(env, orc, frames, policy_seed=2, tag="c0")


@pytest.mark.parametrize("batch", [1, 2], ids=["buckets", "worklist"])
@LANES_AUTO
def test_mixed_modes_tiny_maps_captures_and_resets(lanes, batch):
    """Ragged 1v1 / 2v2 / FFA games on small boards: captures, land transfer, eliminations,
    truncation and auto-reset all happen within a few hundred frames."""
    G = 96
    H, W, mode, P = shapes(G, (3, 9), ((0, 0.34), (1, 0.33), (2, 0.33)), seed=5)
    P = np.where(mode == 2, np.minimum(8, H * W), P).astype(np.int32)
    env, orc = pair(H, W, mode, P, lanes=lanes, seed=11, min_general_dist=1, n_cities=1, max_turns=90)
    env.set_batch_form(batch)
    rollout_policy(env, orc, 300, policy_seed=7, tag="mixed")
    st = env.read_state()[3]
    assert st[:, 2].max() >= 2, "expected several resets"


def test_mixed_modes_no_truncation_long_games():
    G = 40
    H, W, mode, P = shapes(G, (6, 14), ((0, 0.4), (1, 0.3), (2, 0.3)), seed=9)
    env, orc = pair(H, W, mode, P, seed=4, min_general_dist=0, n_cities=-1, city_per_mille=30)
    rollout_policy(env, orc, 250, policy_seed=3, check_every=5, tag="mixed-long")


def test_arbitrary_actions_validation():
    """Random (often illegal or out-of-range) actions through gen_step on both sides."""
    import torch
    G = 64
    H, W, mode, P = shapes(G, (2, 12), ((0, 0.4), (1, 0.3), (2, 0.3)), seed=2)
    P = np.where(mode == 2, np.minimum(P, H * W), P).astype(np.int32)
    env, orc = pair(H, W, mode, P, seed=8, min_general_dist=1, n_cities=2, max_turns=40)
    out = env.new_outputs()
    rng = np.random.default_rng(0)
    for f in range(120):
        rows = random_actions(rng, env.N, 8)
        flat = oracle_actions_flat(env, rows)
        env.step(torch.from_numpy(flat).cuda(), out)
        orc.step(flat_to_rows(env, flat))
        compare_frame(env, out, orc, f"arbitrary frame {f}")


@pytest.mark.parametrize("H,W,mode,P", [(1, 2, 0, 2), (2, 1, 0, 2), (1, 40, 0, 2), (40, 1, 2, 3), (33, 5, 1, 4),
                                        (5, 33, 2, 8), (64, 64, 2, 8), (64, 64, 0, 2), (17, 31, 1, 4),
                                        (3, 3, 2, 8)])
@LANES_AUTO
def test_edge_shapes(H, W, mode, P, lanes):
    G = 6
    env, orc = pair(np.full(G, H), np.full(G, W), np.full(G, mode), np.full(G, P), lanes=lanes,
                    seed=H * 100 + W, min_general_dist=0, n_cities=3, max_turns=25)
    rollout_policy(env, orc, 60, policy_seed=1, check_every=3, tag=f"{H}x{W}")


@LANES_AUTO
def test_no_mountains_and_all_mountains(lanes):
    for thr in (0, 0xFFFFFFFF):
        G = 8
        env, orc = pair(np.full(G, 9), np.full(G, 11), np.zeros(G), np.full(G, 2), lanes=lanes, seed=5,
                        mountain_thresh=thr, n_cities=4, max_turns=30)
        rollout_policy(env, orc, 40, tag=f"mtn{thr}")


def test_two_player_ffa_and_1v1_in_narrow_groups():
    """Two-player free-for-all and 1v1 games step in the two-games-per-warp
    kernels (ragged and uniform shapes) with captures, timeouts and resets."""
    from paper_2606_23348_gb300.generals import GeneralsEnv
    G = 40
    H, W, mode, _ = shapes(G, (4, 24), ((0, 0.5), (2, 0.5)), seed=13)
    P = np.full(G, 2, np.int32)
    env, orc = pair(H, W, mode, P, lanes=2, seed=6, min_general_dist=1, n_cities=3, max_turns=50)
    rollout_policy(env, orc, 120, policy_seed=3, tag="ffa2 ragged")
    kw = dict(seed=9, min_general_dist=2, n_cities=4, max_turns=60)
    env = GeneralsEnv(12, 12, 2, 2, batch=G, **kw)
    env.set_lane_groups(env.LANES_NARROW)
    orc = OracleEnv(np.full(G, 12), np.full(G, 12), np.full(G, 2), np.full(G, 2), **kw)
    rollout_policy(env, orc, 130, policy_seed=5, tag="ffa2 uniform")


def test_reset_subset_and_observe():
    import torch
    G = 20
    H, W, mode, P = shapes(G, (5, 10), ((0, 0.5), (2, 0.5)), seed=3)
    env, orc = pair(H, W, mode, P, seed=2, n_cities=2)
    out = env.new_outputs()
    acts = env.new_actions()
    env.policy(4, acts)
    for f in range(10):
        a = orc.policy(4)
        env.step_policy(acts, out, 4, acts)
        orc.step(a)
    ids = np.array([1, 7, 8, 19], np.int32)
    env.reset(out, torch.from_numpy(ids).cuda())
    orc.reset(ids)
    # reset writes outputs of the listed games only; observe refreshes all
    env.observe(out)
    compare_frame(env, out, orc, "after reset", check_reward=False)
    rw = out.reward.cpu().numpy()
    assert not rw.any() and not out.done.cpu().numpy().any()


def test_state_roundtrip_and_host_step():
    import torch
    from paper_2606_23348_gb300.generals import Outputs
    G = 12
    env, orc = pair(np.full(G, 8), np.full(G, 8), np.zeros(G), np.full(G, 2), seed=9, n_cities=2)
    st = env.read_state()
    env.write_state(*st)
    st2 = env.read_state()
    for x, y in zip(st, st2):
        np.testing.assert_array_equal(x, y)
    out = env.new_outputs()
    h_out = Outputs(env.layout, pin_host=True)
    h_act = torch.zeros(int(env.layout.player_slots), dtype=torch.int32).pin_memory()
    for f in range(15):
        a = orc.policy(3)
        h_act.copy_(torch.from_numpy(oracle_actions_flat(env, a)))
        env.step_host(h_act, h_out)
        orc.step(a)
        compare_frame(env, h_out, orc, f"host step {f}")


@pytest.mark.parametrize("path", golden_io.all_scenarios(), ids=lambda p: p.split("/")[-1][:-4])
def test_golden_scenarios_on_gpu(path):
    """The hand-worked scenarios, loaded into the GPU state and stepped by the kernel."""
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv
    sc = golden_io.load(path)
    P = sc["P"]
    env = GeneralsEnv([sc["H"]], [sc["W"]], [sc["mode"]], [P], seed=7, auto_reset=0, max_turns=sc["max_turns"],
                      n_cities=0, min_general_dist=1)
    army, owner, terrain = sc["board"]
    npad = int(env.npad[0])
    pad = lambda x, v: np.concatenate([x, np.full(npad - x.shape[0], v, x.dtype)])
    alive = sc["alive"] if sc["alive"] is not None else (1 << P) - 1
    scal = np.array([[sc["turn"], 0, 0, alive, 0, 0, 0, 0]], np.uint32)
    env.write_state(pad(army, 0), pad(owner, -1), pad(terrain, 0), scal)
    out = env.new_outputs()
    for k, step in enumerate(sc["steps"]):
        env.step(torch.from_numpy(step["actions"][:P].copy()).cuda(), out)
        torch.cuda.synchronize()
        st = env.read_state()
        a, o, t = env.board(st, 0)
        ea, eo, et = step["board"]
        np.testing.assert_array_equal(t, et)
        np.testing.assert_array_equal(o, eo)
        np.testing.assert_array_equal(a, ea)
        s = st[3][0]
        names = {"turn": 0, "alive": 3, "invalid": 5, "saturated": 6}
        for name, val in step["checks"].items():
            if name in names:
                assert int(s[names[name]]) == val, (name, int(s[names[name]]), val)
            elif name == "done":
                assert int(out.done.cpu()[0]) == val
            elif name == "reward":
                np.testing.assert_array_equal(out.reward.cpu().numpy()[:P], np.array(val, np.float32))
        for p, grids in step["obs"].items():
            for name, grid in grids.items():
                key = {"vis": "obs_vis", "terrain": "obs_terrain", "owner": "obs_owner", "army": "obs_army",
                       "mask": "mask"}[name]
                got = env.plane(getattr(out, key).cpu().numpy(), 0, p).astype(np.int64)
                np.testing.assert_array_equal(got, grid, err_msg=f"{sc['name']} obs {p} {name}")
        if step["scoreboard"] is not None:
            sb = out.scoreboard.cpu().numpy()
            assert sb[:P, 0].tolist() == step["scoreboard"][0]
            assert sb[:P, 1].tolist() == step["scoreboard"][1]


def test_full_size_24x24_65536_sampled():
    """The 65,536-game 24x24 workload in the launch shape the benchmark times:
    every game advances; three blocks of 64 games are replayed by the oracle."""
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv
    H, W, mode, P, gen, _ = workload("1v1-65536x24x24")
    env = GeneralsEnv(H, W, mode, P, seed=1, **gen)
    out = env.new_outputs()
    acts = env.new_actions()
    env.policy(2, acts)
    frames = 24
    hist = []
    for f in range(frames):
        hist.append(acts.cpu().numpy().copy())
        env.step_policy(acts, out, 2, acts)
    torch.cuda.synchronize()
    st = env.read_state()
    assert np.all(st[3][:, 1] == frames) and np.all(st[3][:, 7] == 0)
    for start in (0, 32768 - 32, 65536 - 64):
        n = 64
        orc = OracleEnv(H[start:start + n], W[start:start + n], mode[start:start + n], P[start:start + n], seed=1,
                        game_id_base=start, **gen)
        for f in range(frames):
            a = orc.policy(2)
            np.testing.assert_array_equal(a[:, :2].reshape(-1), hist[f][2 * start:2 * (start + n)])
            orc.step(a)
        for k in range(n):
            g = start + k
            for x, y in zip(env.board(st, g), orc.board(k)):
                np.testing.assert_array_equal(x, y)
            for p in range(2):
                ob = orc.observe(k, p)
                for key, name in (("obs_army", "army"), ("obs_owner", "owner"), ("obs_terrain", "terrain"),
                                  ("obs_vis", "vis"), ("mask", "mask")):
                    o = int(env.plane_off[g]) + p * 576
                    np.testing.assert_array_equal(getattr(out, key)[o:o + 576].cpu().numpy(), ob[name])


@pytest.mark.parametrize("opts", [
    dict(bfs_distance=1),
    dict(bfs_distance=1, max_general_dist=4, min_general_dist=1),
    dict(bfs_distance=1, castle_radius=6),
    dict(bfs_distance=0, castle_radius=6, max_general_dist=9),
    dict(bfs_distance=1, castle_radius=3, max_general_dist=6, mountain_thresh=0x60000000),
], ids=["bfs", "bfs-cap4", "bfs-castle6", "manhattan-castle6-cap9", "bfs-dense-mountains"])
def test_generator_options_match_oracle(opts):
    """Spawn spacing in BFS steps, the curriculum cap and the castle guarantee,
    over mixed modes and sizes, through many resets."""
    G = 64
    H, W, mode, P = shapes(G, (4, 26), ((0, 0.4), (1, 0.3), (2, 0.3)), seed=21)
    P = np.where(mode == 2, np.minimum(P, H * W), P).astype(np.int32)
    kw = dict(seed=17, n_cities=3, max_turns=30, **opts)
    env, orc = pair(H, W, mode, P, **kw)
    rollout_policy(env, orc, 70, policy_seed=5, check_every=2, tag=str(opts))


def test_spawn_range_curriculum_update():
    import torch
    G = 48
    H, W, mode, P = shapes(G, (10, 20), seed=4)
    kw = dict(seed=3, n_cities=4, bfs_distance=1, castle_radius=6)
    env, _ = pair(H, W, mode, P, max_general_dist=4, min_general_dist=1, **kw)
    out = env.new_outputs()
    env.set_spawn_range(2, 9)  # the curriculum widens
    env.reset(out)
    orc = OracleEnv(H, W, mode, P, max_general_dist=9, min_general_dist=2, **kw)
    orc.reset()
    compare_frame(env, out, orc, "after widening", check_reward=False)


def test_full_size_every_game_matches_oracle():
    """All 65,536 games of the 24x24 workload after 12 frames of the fused step +
    policy, every board byte and the scalars, against the oracle run by a spawn
    pool over disjoint game-id ranges on the host cores."""
    import torch
    from oracle.pool import replay_workload
    from paper_2606_23348_gb300.generals import GeneralsEnv
    name = "1v1-65536x24x24"
    H, W, mode, P, gen, _ = workload(name)
    env = GeneralsEnv(H, W, mode, P, seed=1, **gen)
    out = env.new_outputs()
    acts = env.new_actions()
    env.policy(2, acts)
    frames = 12
    for f in range(frames):
        env.step_policy(acts, out, 2, acts)
    torch.cuda.synchronize()
    st = env.read_state()
    boards, scal = replay_workload(name, env.G, 1, 2, frames)
    bad = []
    for g in range(env.G):
        got = env.board(st, g)
        if not all(np.array_equal(x, y) for x, y in zip(got, boards[g])):
            bad.append(g)
        s = st[3][g]
        if (int(s[0]), int(s[1]), int(s[2]), int(s[3])) != tuple(int(x) for x in scal[g]):
            bad.append(g)
    assert not bad, f"{len(bad)} games differ, first {bad[:5]}"


EXHAUSTIVE_POSITIONS = [
    (3, ("6@0G 3@0 0", "M 4@1 2@1", "0 0 5@1G")),
    (3, ("5@0G 45C 0", "3@0 M 9@1", "2@1 0 4@1G")),
    (3, ("2@0G 7@1 3@1G", "2@0 1@1 0", "0 0 M")),
    (4, ("5@0G 3@0 0 M", "2@0 4@1 0 0", "0 M 6@1 2@1", "0 0 3@1 7@1G")),
    (4, ("3@0G 45C 2@0 0", "M 9@1 0 1@0", "4@1 0 M 0", "2@1 0 0 5@1G")),
]


@pytest.mark.parametrize("side,rows", EXHAUSTIVE_POSITIONS, ids=[f"{s}x{s}-{i}" for i, (s, _) in enumerate(
    EXHAUSTIVE_POSITIONS)])
@LANES
def test_exhaustive_joint_actions_on_gpu(side, rows, lanes):
    """Every joint action of both players on a hand-built position, one game
    per joint action in a single launch (81^2 games on 3x3, 144^2 on 4x4),
    at an even and an odd turn, with auto-reset on: every state and output
    byte against the oracle."""
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv
    N = side * side
    army, owner, terrain = golden_io.parse_board(list(rows), side, side)
    A = np.arange(9 * N, dtype=np.int32)
    a0, a1 = np.meshgrid(A, A, indexing="ij")
    acts = np.stack([a0.reshape(-1), a1.reshape(-1)], axis=1)
    G = acts.shape[0]
    for turn in (0, 1):
        kw = dict(seed=9, n_cities=1, min_general_dist=1)
        env = GeneralsEnv(np.full(G, side), np.full(G, side), np.zeros(G), np.full(G, 2), **kw)
        env.set_lane_groups(lanes)
        orc = OracleEnv(np.full(G, side), np.full(G, side), np.zeros(G), np.full(G, 2), **kw)
        npad = int(env.npad[0])
        pad = lambda x, v: np.concatenate([x, np.full(npad - N, v, x.dtype)])
        scal = np.zeros((G, 8), np.uint32)
        scal[:, 0] = turn
        scal[:, 3] = 3
        env.write_state(np.tile(pad(army, 0), G), np.tile(pad(owner, -1), G), np.tile(pad(terrain, 0), G), scal)
        for g in range(G):
            orc.set_game(g, army, owner, terrain, turn=turn)
        out = env.new_outputs()
        env.step(torch.from_numpy(acts.reshape(-1).copy()).cuda(), out)
        rows8 = np.zeros((G, 8), np.int32)
        rows8[:, :2] = acts
        orc.step(rows8)
        compare_frame(env, out, orc, f"{side}x{side} turn {turn}")


def test_host_step_pipelined_matches_device_step():
    """gen_step_host on a batch large enough for its pipelined form (chunks of
    games launched on the caller's stream, outputs copied out on a second
    stream) gives the same bytes as the device-buffer step of a twin batch."""
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv, Outputs
    G = 16384 + 7  # chunks of unequal size
    kw = dict(seed=21, n_cities=4)
    host = GeneralsEnv(17, 19, 0, 2, batch=G, **kw)
    dev = GeneralsEnv(17, 19, 0, 2, batch=G, **kw)
    h_out = Outputs(host.layout, pin_host=True)
    d_out = dev.new_outputs()
    acts = dev.new_actions()
    dev.policy(4, acts)
    h_act = acts.cpu().pin_memory()
    h_next = torch.empty_like(h_act).pin_memory()
    for f in range(6):
        host.step_host(h_act, h_out, 4, h_next)
        dev.step_policy(acts, d_out, 4, acts)
        torch.cuda.synchronize()
        for name, ht, dt in zip(("army", "owner", "terrain", "vis", "mask", "reward", "scoreboard", "done"),
                                h_out.tensors(), d_out.tensors()):
            assert torch.equal(ht, dt.cpu()), f"frame {f}: {name}"
        assert torch.equal(h_next, acts.cpu()), f"frame {f}: next actions"
        h_act.copy_(h_next)


def test_two_shards_concatenate_to_one_batch():
    """Replicas with disjoint game ids (the multi-GPU partition): two
    environments holding games [0, G) and [G, 2G) with game_id_base 0 and G
    produce, concatenated, exactly the bytes of one environment of all 2G
    games, which matches the oracle."""
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv
    G = 40
    H, W, mode, P = shapes(2 * G, (5, 16), ((0, 0.4), (1, 0.3), (2, 0.3)), seed=31)
    kw = dict(seed=8, min_general_dist=1, n_cities=2, max_turns=25)
    full = GeneralsEnv(H, W, mode, P, **kw)
    parts = [GeneralsEnv(H[:G], W[:G], mode[:G], P[:G], game_id_base=0, **kw),
             GeneralsEnv(H[G:], W[G:], mode[G:], P[G:], game_id_base=G, **kw)]
    orc = OracleEnv(H, W, mode, P, **kw)
    envs = [full] + parts
    outs = [e.new_outputs() for e in envs]
    acts = [e.new_actions() for e in envs]
    for e, a in zip(envs, acts):
        e.policy(5, a)
    for f in range(50):
        a_orc = orc.policy(5)
        for e, o, a in zip(envs, outs, acts):
            e.step_policy(a, o, 5, a)
        orc.step(a_orc)
    torch.cuda.synchronize()
    for k, t in enumerate(outs[0].tensors()):
        cat = torch.cat([outs[1].tensors()[k], outs[2].tensors()[k]])
        assert torch.equal(t, cat), f"output array {k}"
    assert torch.equal(acts[0], torch.cat(acts[1:]))
    st = [e.read_state() for e in envs]
    for k in range(4):
        np.testing.assert_array_equal(st[0][k], np.concatenate([st[1][k], st[2][k]]))
    compare_frame(full, outs[0], orc, "full batch vs oracle")
