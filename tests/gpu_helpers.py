"""Helpers of the GPU parity tests: run the CUDA path and the oracle side by
side and compare every state and output byte.

Only layout marshalling lives here (placing the oracle's per-game planes at
the library's offsets, with the padding values the header documents); no
rule is computed.
"""
from __future__ import annotations

import numpy as np

PAD = {"obs_army": 0, "obs_owner": -2, "obs_terrain": 4, "obs_vis": 0, "mask": 0}
PLANES = ("obs_army", "obs_owner", "obs_terrain", "obs_vis", "mask")
ORC_NAME = {"obs_army": "army", "obs_owner": "owner", "obs_terrain": "terrain", "obs_vis": "vis", "mask": "mask"}
DTYPES = {"obs_army": np.int16, "obs_owner": np.int8, "obs_terrain": np.int8, "obs_vis": np.uint8,
          "mask": np.uint8}


def oracle_flat_outputs(env, orc, games=None):
    """The oracle's observations in the library's flat layout (all games, or a subset)."""
    pc = int(env.layout.plane_cells)
    flat = {k: np.full(pc, PAD[k], DTYPES[k]) for k in PLANES}
    games = range(env.G) if games is None else games
    for g in games:
        for p in range(int(env.P[g])):
            ob = orc.observe(g if orc.G == env.G else g - games[0], p)
            o = int(env.plane_off[g]) + p * int(env.npad[g])
            n = int(env.N[g])
            for k in PLANES:
                flat[k][o:o + n] = ob[ORC_NAME[k]]
    return flat


def compare_frame(env, out, orc, tag="", check_outputs=True, check_reward=True):
    """Assert bit-exact equality of state, scalars and outputs of every game."""
    import torch
    torch.cuda.synchronize()
    st = env.read_state()
    scal = st[3]
    for g in range(env.G):
        a, o, t = env.board(st, g)
        ea, eo, et = orc.board(g)
        if not (np.array_equal(t, et) and np.array_equal(o, eo) and np.array_equal(a, ea)):
            bad = np.flatnonzero((a != ea) | (o != eo) | (t != et))[:5]
            raise AssertionError(f"{tag} game {g}: board differs at cells {bad.tolist()}: gpu "
                                 f"{list(zip(a[bad], o[bad], t[bad]))} oracle {list(zip(ea[bad], eo[bad], et[bad]))}")
        s = orc.scalars(g)
        got = dict(turn=scal[g, 0], frame=scal[g, 1], epoch=scal[g, 2], alive=scal[g, 3], finished=scal[g, 4],
                   invalid=scal[g, 5], saturated=scal[g, 6])
        for k, v in got.items():
            assert int(v) == s[k], f"{tag} game {g}: {k} gpu {int(v)} oracle {s[k]}"
        assert scal[g, 7] == 0, f"{tag} game {g}: device error word {scal[g, 7]}"
    if not check_outputs:
        return
    flat = oracle_flat_outputs(env, orc)
    for k in PLANES:
        got = getattr(out, k).cpu().numpy()
        if not np.array_equal(got, flat[k]):
            i = int(np.flatnonzero(got != flat[k])[0])
            g = int(np.searchsorted(env.plane_off, i, side="right") - 1)
            raise AssertionError(f"{tag} plane {k}: first difference at element {i} (game {g}): gpu {got[i]} "
                                 f"oracle {flat[k][i]}")
    sb = out.scoreboard.cpu().numpy()
    rw = out.reward.cpu().numpy()
    dn = out.done.cpu().numpy()
    for g in range(env.G):
        land, arm = orc.scoreboard(g)
        s = orc.scalars(g)
        o = int(env.player_off[g])
        P = int(env.P[g])
        assert np.array_equal(sb[o:o + P, 0], land[:P]), f"{tag} game {g}: land"
        assert np.array_equal(sb[o:o + P, 1], arm[:P]), f"{tag} game {g}: army"
        if check_reward:
            assert np.array_equal(rw[o:o + P], s["reward"][:P]), f"{tag} game {g}: reward {rw[o:o + P]} vs {s['reward'][:P]}"
            assert int(dn[g]) == s["done"], f"{tag} game {g}: done {dn[g]} vs {s['done']}"


def oracle_actions_flat(env, acts8):
    """[G][8] oracle action rows -> the library's flat per-player slots."""
    flat = np.zeros(int(env.layout.player_slots), np.int32)
    for g in range(env.G):
        o = int(env.player_off[g])
        flat[o:o + int(env.P[g])] = acts8[g, :int(env.P[g])]
    return flat


def flat_to_rows(env, flat):
    rows = np.zeros((env.G, 8), np.int32)
    for g in range(env.G):
        o = int(env.player_off[g])
        rows[g, :int(env.P[g])] = flat[o:o + int(env.P[g])]
    return rows
