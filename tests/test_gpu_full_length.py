"""The full-length configurations, as the benchmark's workloads define them,
on the GPU and against the oracle on sampled games: the default workload's
65,536 1v1 games on 24x24 for 2,000 frames and the mixed batch's 32,768
games (1v1, 2v2, 8-player free-for-all, sides 20..40) for 1,000 frames, one
step + policy launch per frame, auto-reset on.  Blocks of games spread over
the batch are replayed by the oracle for the whole run; their boards,
counters (turn, frame, epoch, alive players, invalid actions, saturations),
last-frame outputs and next actions must match byte for byte.  Under the
benchmark policy few games end within these runs (none of the first 256 of
the default workload in 2,000 frames), so each workload runs once more with
a turn limit that regenerates every game along the way."""
import numpy as np
import pytest

from oracle import OracleEnv
from paper_2606_23348_gb300.workloads import workload

pytestmark = pytest.mark.gpu

PLANES = (("obs_army", "army"), ("obs_owner", "owner"), ("obs_terrain", "terrain"), ("obs_vis", "vis"),
          ("mask", "mask"))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_23348_gb300.build import build_library
    build_library()


def _run_and_replay(name, frames, blocks, n, policy_seed=2, max_turns=0):
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv
    H, W, mode, P, gen, _ = workload(name)
    if max_turns:
        gen = dict(gen, max_turns=max_turns)
    env = GeneralsEnv(H, W, mode, P, seed=1, **gen)
    out, acts = env.new_outputs(), env.new_actions()
    env.policy(policy_seed, acts)
    for _ in range(frames):
        env.step_policy(acts, out, policy_seed, acts)
    torch.cuda.synchronize()
    state = env.read_state()
    got_acts = acts.cpu().numpy()
    planes = {k: getattr(out, k).cpu().numpy() for k, _ in PLANES}
    done = out.done.cpu().numpy()
    epochs = state[3][:, 2]
    if max_turns:
        assert epochs.min() >= 1, f"every game should reach the {max_turns}-turn limit within {frames} frames"
    if epochs.max() >= 1:  # one more block starting at the first regenerated game
        blocks = tuple(blocks) + (min(int(np.flatnonzero(epochs >= 1)[0]), env.G - n),)
    for start in blocks:
        orc = OracleEnv(H[start:start + n], W[start:start + n], mode[start:start + n], P[start:start + n],
                        game_id_base=start, seed=1, **gen)
        for _ in range(frames):
            orc.step(orc.policy(policy_seed))
        nxt = orc.policy(policy_seed)
        for i in range(n):
            g = start + i
            for x, y in zip(env.board(state, g), orc.board(i)):
                np.testing.assert_array_equal(x, y, err_msg=f"game {g}: board after {frames} frames")
            s = orc.scalars(i)
            sc = state[3][g]
            assert [int(v) for v in sc[:7]] == [s["turn"], s["frame"], s["epoch"], s["alive"], s["finished"],
                                                s["invalid"], s["saturated"]], f"game {g}: counters"
            assert sc[7] == 0, f"game {g}: device error word"
            assert int(done[g]) == s["done"], f"game {g}: done"
            for p in range(int(env.P[g])):
                ob = orc.observe(i, p)
                o = int(env.plane_off[g]) + p * int(env.npad[g])
                for key, oname in PLANES:
                    np.testing.assert_array_equal(planes[key][o:o + int(env.N[g])], ob[oname],
                                                  err_msg=f"game {g} player {p}: {key}")
            po = int(env.player_off[g])
            np.testing.assert_array_equal(got_acts[po:po + int(env.P[g])], nxt[i, :int(env.P[g])],
                                          err_msg=f"game {g}: next actions")


def test_default_workload_2000_frames_sampled():
    """65,536 x 24x24 1v1, 2,000 frames with auto-reset, four blocks of 8 games."""
    _run_and_replay("1v1-65536x24x24", 2000, (0, 21840, 43690, 65536 - 8), 8)


def test_mixed_workload_1000_frames_sampled():
    """32,768 mixed games, 1,000 frames with auto-reset, four blocks of 6 games."""
    _run_and_replay("mixed-32768-sides20to40", 1000, (0, 10922, 21845, 32768 - 6), 6)


def test_default_workload_2000_frames_with_turn_limit_sampled():
    """The same run with a 300-turn limit: every game is regenerated several times."""
    _run_and_replay("1v1-65536x24x24", 2000, (0, 21840, 43690, 65536 - 8), 8, max_turns=300)


def test_mixed_workload_1000_frames_with_turn_limit_sampled():
    """The mixed run with a 200-turn limit: the last of the 1,000 frames is a
    regeneration frame (done set, outputs of the fresh maps)."""
    _run_and_replay("mixed-32768-sides20to40", 1000, (0, 10922, 21845, 32768 - 6), 6, max_turns=200)
