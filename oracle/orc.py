"""ctypes binding of the C oracle (test infrastructure only).

The oracle is compiled from ``generals_oracle.c`` with the host C compiler
into ``oracle/_build/``.  Nothing here computes game rules: every rule is in
the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "generals_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

MAXP = 8


class OracleParams(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64),
        ("game_id_base", C.c_uint64),
        ("mountain_thresh", C.c_uint32),
        ("n_cities", C.c_int32),
        ("city_per_mille", C.c_int32),
        ("city_army_min", C.c_int32),
        ("city_army_max", C.c_int32),
        ("min_general_dist", C.c_int32),
        ("max_turns", C.c_int32),
        ("auto_reset", C.c_int32),
        ("max_general_dist", C.c_int32),
        ("bfs_distance", C.c_int32),
        ("castle_radius", C.c_int32),
    ]


def build_oracle(force: bool = False) -> str:
    """Compile the oracle shared object (plain C, -O2) and return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def oracle_lib():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build_oracle())
            P = C.POINTER
            lib.orc_sm.restype = C.c_uint64
            lib.orc_sm.argtypes = [C.c_uint64, C.c_uint64]
            lib.orc_key.restype = C.c_uint64
            lib.orc_key.argtypes = [C.c_uint64] * 4
            lib.orc_draw.restype = C.c_uint32
            lib.orc_draw.argtypes = [C.c_uint64, C.c_uint64]
            lib.orc_env_new.restype = C.c_int
            lib.orc_env_new.argtypes = [P(C.c_void_p), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        P(OracleParams)]
            lib.orc_env_free.argtypes = [C.c_void_p]
            lib.orc_reset.restype = C.c_int
            lib.orc_reset.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
            lib.orc_step.argtypes = [C.c_void_p, C.c_void_p]
            lib.orc_observe_player.argtypes = [C.c_void_p, C.c_int32, C.c_int32] + [C.c_void_p] * 5
            lib.orc_get_scoreboard.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]
            lib.orc_policy.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p]
            lib.orc_get_scalars.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]
            lib.orc_get_board.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
            lib.orc_set_game.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                         C.c_uint32, C.c_uint32, C.c_uint32]
            lib.orc_feat_new.restype = C.c_int
            lib.orc_feat_new.argtypes = [P(C.c_void_p), C.c_void_p, C.c_int32, C.c_int32]
            lib.orc_feat_free.argtypes = [C.c_void_p]
            lib.orc_feat_build.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            lib.orc_sample_actions.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]
            lib.orc_exp37.restype = C.c_float
            lib.orc_exp37.argtypes = [C.c_float]
            _lib = lib
    return _lib


def sm(seed: int, n: int) -> int:
    return int(oracle_lib().orc_sm(seed, n))


def key(seed: int, a: int, b: int, c: int) -> int:
    return int(oracle_lib().orc_key(seed, a, b, c))


def draw(k: int, i: int) -> int:
    return int(oracle_lib().orc_draw(k, i))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def players_for(mode: int, n_players: int) -> int:
    return 2 if mode == 0 else 4 if mode == 1 else int(n_players)


class OracleEnv:
    """A batch of games held by the oracle.

    ``H``, ``W``, ``mode``, ``n_players`` are per-game integer arrays.
    """

    def __init__(self, H, W, mode, n_players, *, seed=1, game_id_base=0, mountain_thresh=858993459,
                 n_cities=8, city_per_mille=0, city_army_min=40, city_army_max=50, min_general_dist=0,
                 max_turns=0, auto_reset=1, max_general_dist=0, bfs_distance=0, castle_radius=0):
        self.lib = oracle_lib()
        self.H = np.ascontiguousarray(H, dtype=np.int32)
        self.W = np.ascontiguousarray(W, dtype=np.int32)
        self.mode = np.ascontiguousarray(mode, dtype=np.int32)
        self.n_players = np.ascontiguousarray(n_players, dtype=np.int32)
        self.G = int(self.H.shape[0])
        self.P = np.array([players_for(m, n) for m, n in zip(self.mode, self.n_players)], dtype=np.int32)
        self.N = (self.H * self.W).astype(np.int64)
        self.params = OracleParams(seed, game_id_base, mountain_thresh, n_cities, city_per_mille, city_army_min,
                                   city_army_max, min_general_dist, max_turns, auto_reset, max_general_dist,
                                   bfs_distance, castle_radius)
        h = C.c_void_p()
        rc = self.lib.orc_env_new(C.byref(h), self.G, _ptr(self.H), _ptr(self.W), _ptr(self.mode),
                                  _ptr(self.n_players), C.byref(self.params))
        if rc != 0:
            raise ValueError(f"orc_env_new failed ({rc})")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.orc_env_free(self.h)
            self.h = None

    def __del__(self):
        self.close()

    # ---- stepping -------------------------------------------------------
    def step(self, actions: np.ndarray):
        a = np.zeros((self.G, MAXP), dtype=np.int32)
        actions = np.asarray(actions, dtype=np.int32)
        a[:, : actions.shape[1]] = actions
        self.lib.orc_step(self.h, _ptr(a))

    def reset(self, game_ids=None):
        if game_ids is None:
            rc = self.lib.orc_reset(self.h, None, 0)
        else:
            ids = np.ascontiguousarray(game_ids, dtype=np.int32)
            rc = self.lib.orc_reset(self.h, _ptr(ids), int(ids.shape[0]))
        if rc != 0:
            raise ValueError("orc_reset: bad game id")

    def policy(self, policy_seed: int) -> np.ndarray:
        a = np.zeros((self.G, MAXP), dtype=np.int32)
        self.lib.orc_policy(self.h, policy_seed, _ptr(a))
        return a

    # ---- inspection -----------------------------------------------------
    def board(self, g: int):
        n = int(self.N[g])
        army = np.zeros(n, np.int16)
        owner = np.zeros(n, np.int8)
        terrain = np.zeros(n, np.int8)
        self.lib.orc_get_board(self.h, g, _ptr(army), _ptr(owner), _ptr(terrain))
        return army, owner, terrain

    def scalars(self, g: int) -> dict:
        s = np.zeros(16, np.int64)
        r = np.zeros(8, np.float32)
        self.lib.orc_get_scalars(self.h, g, _ptr(s), _ptr(r))
        return {"turn": int(s[0]), "frame": int(s[1]), "epoch": int(s[2]), "alive": int(s[3]),
                "finished": int(s[4]), "invalid": int(s[5]), "saturated": int(s[6]), "done": int(s[7]),
                "gpos": [int(x) for x in s[8:16]], "reward": r.copy()}

    def observe(self, g: int, p: int):
        n = int(self.N[g])
        army = np.zeros(n, np.int16)
        owner = np.zeros(n, np.int8)
        terrain = np.zeros(n, np.int8)
        vis = np.zeros(n, np.uint8)
        mask = np.zeros(n, np.uint8)
        self.lib.orc_observe_player(self.h, g, p, _ptr(army), _ptr(owner), _ptr(terrain), _ptr(vis), _ptr(mask))
        return {"army": army, "owner": owner, "terrain": terrain, "vis": vis, "mask": mask}

    def scoreboard(self, g: int):
        land = np.zeros(8, np.int32)
        army = np.zeros(8, np.int32)
        self.lib.orc_get_scoreboard(self.h, g, _ptr(land), _ptr(army))
        return land, army

    def sample_actions(self, logits, seed: int):
        """Sample one action per player from per-game [P][N * 9] float32 logits
        (a list over games).  Returns (actions [G][8] int32, list over games
        of [P][N * 9] uint8 legal-entry masks)."""
        flat = np.ascontiguousarray(np.concatenate([np.asarray(l, np.float32).reshape(-1) for l in logits]))
        mask = np.zeros(flat.shape[0], np.uint8)
        acts = np.zeros((self.G, MAXP), np.int32)
        self.lib.orc_sample_actions(self.h, _ptr(flat), int(seed), _ptr(acts), _ptr(mask))
        res, off = [], 0
        for P, N in zip(self.P, self.N):
            n = int(P) * 9 * int(N)
            res.append(mask[off:off + n].reshape(int(P), 9 * int(N)))
            off += n
        return acts, res

    def set_game(self, g: int, army, owner, terrain, *, turn=0, alive=None, frame=0, epoch=0):
        army = np.ascontiguousarray(army, np.int16)
        owner = np.ascontiguousarray(owner, np.int8)
        terrain = np.ascontiguousarray(terrain, np.int8)
        assert army.shape[0] == self.N[g]
        if alive is None:
            alive = (1 << int(self.P[g])) - 1
        self.lib.orc_set_game(self.h, g, _ptr(army), _ptr(owner), _ptr(terrain), int(turn), int(alive),
                              int(frame), int(epoch))


class OracleFeatures:
    """Feature tensor builder over an OracleEnv (Appendix A): C = 24 + 2 * hist
    channels per player.  ``build()`` folds the current frame into each
    player's memory and returns a list over games of [P][C][N] float32;
    ``series`` then holds, per game, [P][window][2] int32 (opponents' army,
    land; newest first) when ``window`` > 0."""

    def __init__(self, env: OracleEnv, hist: int = 7, window: int = 0):
        self.env = env
        self.lib = env.lib
        self.hist = int(hist)
        self.window = int(window)
        self.C = 24 + 2 * self.hist
        self.series = None
        h = C.c_void_p()
        if self.lib.orc_feat_new(C.byref(h), env.h, self.hist, self.window) != 0:
            raise ValueError("orc_feat_new failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.orc_feat_free(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def build(self):
        sizes = [int(P) * self.C * int(N) for P, N in zip(self.env.P, self.env.N)]
        out = np.zeros(int(sum(sizes)), np.float32)
        ser = np.zeros(int(sum(self.env.P)) * 2 * max(self.window, 1), np.int32)
        self.lib.orc_feat_build(self.h, _ptr(out), _ptr(ser) if self.window > 0 else None)
        if self.window > 0:
            self.series, soff = [], 0
            for P in self.env.P:
                n = int(P) * 2 * self.window
                self.series.append(ser[soff:soff + n].reshape(int(P), self.window, 2))
                soff += n
        res, off = [], 0
        for (P, N), n in zip(zip(self.env.P, self.env.N), sizes):
            res.append(out[off:off + n].reshape(int(P), self.C, int(N)))
            off += n
        return res


def exp37(x: float) -> float:
    """The reproducible single-precision exponential used by the sampler."""
    return float(oracle_lib().orc_exp37(float(x)))
