"""Multi-frame rollouts (resident, CUDA graph, plain launches) vs the oracle,
and size-bucketed ragged batches, bit-exact frame by frame."""
import types

import numpy as np
import pytest

from gpu_helpers import PLANES, compare_frame, oracle_actions_flat
from oracle import OracleEnv
from paper_2606_23348_gb300.workloads import shapes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_23348_gb300.build import build_library
    build_library()


def frame_view(env, out, k):
    """Frame k of a multi-frame Outputs as a one-frame object."""
    pc, ps, G = int(env.layout.plane_cells), int(env.layout.player_slots), env.G
    v = types.SimpleNamespace()
    for name in PLANES:
        setattr(v, name, getattr(out, name)[k * pc:(k + 1) * pc])
    v.reward = out.reward[k * ps:(k + 1) * ps]
    v.scoreboard = out.scoreboard[k * ps:(k + 1) * ps]
    v.done = out.done[k * G:(k + 1) * G]
    return v


def make_pair(G=48, seed=3, two_player=False, lanes=0, batch=0):
    from paper_2606_23348_gb300.generals import GeneralsEnv
    modes = ((0, 0.5), (2, 0.5)) if two_player else ((0, 0.4), (1, 0.3), (2, 0.3))
    H, W, mode, P = shapes(G, (4, 20), modes, seed=seed)
    P = np.where(mode == 2, np.minimum(P, H * W), P).astype(np.int32)
    if two_player:
        P = np.full(G, 2, np.int32)
    kw = dict(seed=seed, min_general_dist=1, n_cities=2, max_turns=40)
    env = GeneralsEnv(H, W, mode, P, **kw)
    if lanes:
        env.set_lane_groups(lanes)
    if batch:
        env.set_batch_form(batch)
    return env, OracleEnv(H, W, mode, P, **kw)


# a batch of several size buckets: one launch per bucket, or one work-list launch
BATCH = pytest.mark.parametrize("batch", [1, 2], ids=["buckets", "worklist"])


@BATCH
@pytest.mark.parametrize("lanes", [0, 2], ids=["auto", "narrow"])
@pytest.mark.parametrize("form", [0, 1, 2], ids=["resident", "graph", "launches"])
def test_rollout_matches_oracle(form, lanes, batch):
    env, orc = make_pair(lanes=lanes, batch=batch)
    assert len(set(zip(env.npad // 256, env.P))) > 1  # several size buckets
    check_rollout(env, orc, form)


@pytest.mark.parametrize("form", [0, 1, 2], ids=["resident", "graph", "launches"])
def test_rollout_two_player_ffa_with_1v1(form):
    """Two-player free-for-all games share the narrow lane groups (two or
    four games per warp) with 1v1 games: the same rules, bit-exact."""
    env, orc = make_pair(G=64, seed=17, two_player=True, lanes=2)
    assert set(env.P.tolist()) == {2} and max(env.npad) <= 576
    check_rollout(env, orc, form)


@pytest.mark.parametrize("lanes", [1, 2], ids=["warp", "narrow"])
@pytest.mark.parametrize("mode,P", [(0, 2), (1, 4)], ids=["1v1", "2v2"])
@pytest.mark.parametrize("form", [0, 1, 2], ids=["resident", "graph", "launches"])
def test_uniform_batch_rollout_matches_oracle(form, mode, P, lanes):
    """A batch of one board shape runs the uniform-shape kernels: every frame
    of each form against the oracle, with a warp per game and (1v1) two or
    four games per warp."""
    from paper_2606_23348_gb300.generals import GeneralsEnv
    G = 64
    kw = dict(seed=21, min_general_dist=1, n_cities=4, max_turns=30)
    env = GeneralsEnv(12, 13, mode, P, batch=G, **kw)
    env.set_lane_groups(lanes)
    orc = OracleEnv(np.full(G, 12), np.full(G, 13), np.full(G, mode), np.full(G, P), **kw)
    check_rollout(env, orc, form)


@pytest.mark.parametrize("form", [0, 1], ids=["resident", "graph"])
def test_uniform_batch_rollout_two_per_warp_large_boards(form):
    """Uniform 28x30 1v1 boards (840 cells: too many for four games per warp,
    two per warp in multi-frame launches too) against the oracle."""
    from paper_2606_23348_gb300.generals import GeneralsEnv
    G = 40
    kw = dict(seed=23, min_general_dist=2, n_cities=6, max_turns=24)
    env = GeneralsEnv(28, 30, 0, 2, batch=G, **kw)
    env.set_lane_groups(env.LANES_NARROW)
    orc = OracleEnv(np.full(G, 28), np.full(G, 30), np.zeros(G), np.full(G, 2), **kw)
    check_rollout(env, orc, form)


def check_rollout(env, orc, form):
    import torch
    K = 9
    out = env.new_outputs(frames=K)
    acts = env.new_actions()
    log = torch.zeros(K * int(env.layout.player_slots), dtype=torch.int32, device="cuda")
    env.policy(5, acts)
    for rep in range(3):  # the graph form replays from the second call on
        env.rollout(K, 5, acts, out, log, form)
        torch.cuda.synchronize()
        logs = log.cpu().numpy().reshape(K, -1)
        for k in range(K):
            a = orc.policy(5)
            np.testing.assert_array_equal(logs[k], oracle_actions_flat(env, a), err_msg=f"rep {rep} frame {k}")
            orc.step(a)
            if k < K - 1:
                # state is only comparable at the end; outputs every frame
                from gpu_helpers import oracle_flat_outputs
                flat = oracle_flat_outputs(env, orc)
                fv = frame_view(env, out, k)
                for name in PLANES:
                    np.testing.assert_array_equal(getattr(fv, name).cpu().numpy(), flat[name],
                                                  err_msg=f"rep {rep} frame {k} {name}")
        compare_frame(env, frame_view(env, out, K - 1), orc, f"rep {rep} last frame")
        np.testing.assert_array_equal(acts.cpu().numpy(), oracle_actions_flat(env, orc.policy(5)))


def test_rollout_forms_agree_on_full_workload_slice():
    """The three rollout forms, each with one launch per size bucket and with
    the work-list launch, give identical bytes on a ragged 15..30 batch."""
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv
    H, W, mode, P = shapes(4096, (15, 30), seed=7)
    res = []
    for form, batch in ((0, 2), (1, 2), (2, 2), (0, 1), (1, 1), (2, 1)):
        env = GeneralsEnv(H, W, mode, P, seed=7, n_cities=-1, city_per_mille=20)
        env.set_batch_form(batch)
        out = env.new_outputs(frames=4)
        acts = env.new_actions()
        env.policy(9, acts)
        env.rollout(4, 9, acts, out, None, form)
        env.rollout(4, 9, acts, out, None, form)
        torch.cuda.synchronize()
        res.append([t.cpu().numpy().copy() for t in out.tensors()] + [acts.cpu().numpy().copy()])
    for other in res[1:]:
        for x, y in zip(res[0], other):
            np.testing.assert_array_equal(x, y)


def test_autotune_keeps_results():
    import torch
    env, orc = make_pair(G=40, seed=11)
    rep = env.autotune(steps=2)
    assert "bucket" in rep
    out = env.new_outputs()
    acts = env.new_actions()
    env.policy(3, acts)
    for f in range(10):
        a = orc.policy(3)
        env.step_policy(acts, out, 3, acts)
        orc.step(a)
    compare_frame(env, out, orc, "after autotune")


def test_tuned_and_default_shapes_give_identical_bytes():
    """Every choice the autotuner makes (games per warp, batch form, the
    rollout form AUTO runs, sampler form, feature-builder form, games per
    CTA) leaves the results as they were: a tuned and an untuned environment
    of the same games agree byte for byte on rollouts, sampled actions and
    the feature tensor."""
    import torch
    from paper_2606_23348_gb300.generals import ROLLOUT_AUTO, ROLLOUT_RESIDENT
    tuned, _ = make_pair(G=64, seed=23)
    plain, _ = make_pair(G=64, seed=23)
    rep = tuned.autotune(steps=2)
    assert "lanes:" in rep and "batch:" in rep and "rollout" in rep and "sampler:" in rep
    fa, fb = tuned.features(7, 16), plain.features(7, 16)
    xa, xb = fa.new_output(), fb.new_output()
    fa.autotune(xa, steps=2)  # folds the first frame, as this build does on the other side
    fb.build(xb)
    g = torch.Generator(device="cuda").manual_seed(5)
    logits = torch.randn(int(tuned.layout.plane_cells) * 9, generator=g, device="cuda")
    res = []
    for env, fbld, x, form in ((tuned, fa, xa, ROLLOUT_AUTO), (plain, fb, xb, ROLLOUT_RESIDENT)):
        out = env.new_outputs(frames=6)
        acts = env.new_actions()
        env.policy(4, acts)
        env.rollout(6, 4, acts, out, None, form)
        env.rollout(6, 4, acts, out, None, form)
        sampled = env.sample_actions(logits, 9)
        fbld.build(x)
        torch.cuda.synchronize()
        res.append([t.cpu().numpy().copy() for t in out.tensors()] + [acts.cpu().numpy(), sampled.cpu().numpy(),
                                                                      x.cpu().numpy()])
    for i, (u, v) in enumerate(zip(*res)):
        np.testing.assert_array_equal(u, v, err_msg=f"array {i}")


def _check_sampled(env, out, K, H, W, mode, P, gen, blocks, n, policy_seed, log=None):
    """Replay sampled blocks of games in the oracle and compare every frame of the rollout buffer."""
    import torch
    pc, ps = int(env.layout.plane_cells), int(env.layout.player_slots)
    for start in blocks:
        orc = OracleEnv(H[start:start + n], W[start:start + n], mode[start:start + n], P[start:start + n],
                        game_id_base=start, seed=1, **gen)
        for k in range(K):
            a = orc.policy(policy_seed)
            orc.step(a)
            for i in range(n):
                g = start + i
                for p in range(int(env.P[g])):
                    ob = orc.observe(i, p)
                    o = k * pc + int(env.plane_off[g]) + p * int(env.npad[g])
                    nc = int(env.N[g])
                    for key, name in (("obs_army", "army"), ("obs_owner", "owner"), ("obs_terrain", "terrain"),
                                      ("obs_vis", "vis"), ("mask", "mask")):
                        got = getattr(out, key)[o:o + nc].cpu().numpy()
                        np.testing.assert_array_equal(got, ob[name], err_msg=f"frame {k} game {g} p{p} {key}")
                s = orc.scalars(i)
                assert int(out.done[k * env.G + g].cpu()) == s["done"]
                if log is not None:
                    so = k * ps + int(env.player_off[g])
                    np.testing.assert_array_equal(log[so:so + int(env.P[g])].cpu().numpy(), a[i, :int(env.P[g])])


def test_full_size_ragged_131072_resident_64_frames_sampled():
    """The ragged 131,072-game workload in the form the benchmark times: one
    resident 64-frame rollout; three blocks of 24 games replayed by the oracle."""
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv
    from paper_2606_23348_gb300.workloads import workload
    H, W, mode, P, gen, _ = workload("1v1-131072-ragged15to30")
    env = GeneralsEnv(H, W, mode, P, seed=1, **gen)
    K = 64
    out = env.new_outputs(frames=K)
    acts = env.new_actions()
    log = torch.zeros(K * int(env.layout.player_slots), dtype=torch.int32, device="cuda")
    env.policy(2, acts)
    env.rollout(K, 2, acts, out, log, 0)
    torch.cuda.synchronize()
    _check_sampled(env, out, K, H, W, mode, P, gen, (0, 65536 - 12, 131072 - 24), 24, 2, log)


def test_full_size_24x24_65536_resident_64_frames_sampled():
    """The default workload in the form the benchmark's resident figure
    times: one 64-frame rollout of 65,536 games of one shape (four games per
    warp); three blocks of 24 games replayed by the oracle."""
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv
    from paper_2606_23348_gb300.workloads import workload
    H, W, mode, P, gen, _ = workload("1v1-65536x24x24")
    env = GeneralsEnv(H, W, mode, P, seed=1, **gen)
    K = 64
    out = env.new_outputs(frames=K)
    acts = env.new_actions()
    log = torch.zeros(K * int(env.layout.player_slots), dtype=torch.int32, device="cuda")
    env.policy(2, acts)
    env.rollout(K, 2, acts, out, log, 0)
    torch.cuda.synchronize()
    _check_sampled(env, out, K, H, W, mode, P, gen, (0, 32768 - 12, 65536 - 24), 24, 2, log)


def test_full_size_mixed_32768_sampled():
    """The mixed 32,768-game workload (1v1 / 2v2 / FFA-8, sides 20..40, 15 size
    buckets) stepped frame by frame; three blocks of 16 games replayed."""
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv
    from paper_2606_23348_gb300.workloads import workload
    H, W, mode, P, gen, _ = workload("mixed-32768-sides20to40")
    env = GeneralsEnv(H, W, mode, P, seed=1, **gen)
    K = 12
    out = env.new_outputs(frames=K)
    acts = env.new_actions()
    env.policy(2, acts)
    env.rollout(K, 2, acts, out, None, 2)  # plain launches, one per bucket per frame
    torch.cuda.synchronize()
    _check_sampled(env, out, K, H, W, mode, P, gen, (0, 16384, 32768 - 16), 16, 2)
