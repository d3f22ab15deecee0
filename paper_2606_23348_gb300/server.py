"""Python binding of the env server (gen_server_* in include/generals.h).

Argument marshalling only: the server, its scheduler thread and every game
step live in libgenerals.  Steps block in C with the GIL released, so Python
threads can act as concurrent clients.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .generals import GenLayoutInfo, GenOutputs, GenParams, default_params, load_library


class ServerConfig(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("max_games", C.c_int64), ("max_cells", C.c_int64),
                ("max_plane_cells", C.c_int64), ("host_outputs", C.c_int32), ("policy_seed", C.c_uint64)]


class ServerStats(C.Structure):
    _fields_ = [("requests", C.c_uint64), ("frames", C.c_uint64), ("ticks", C.c_uint64),
                ("sessions_open", C.c_uint64), ("sessions_admitted", C.c_uint64), ("sessions_waited", C.c_uint64),
                ("seconds", C.c_double), ("frames_per_s", C.c_double), ("lat_p50_ms", C.c_double),
                ("lat_p99_ms", C.c_double), ("lat_mean_ms", C.c_double), ("tick_games_mean", C.c_double),
                ("bytes_in_use", C.c_double), ("budget", C.c_double), ("sessions_waited_budget", C.c_uint64),
                ("peak_bytes_in_use", C.c_double), ("service_p50_ms", C.c_double), ("service_p99_ms", C.c_double),
                ("offered_requests_per_s", C.c_double), ("tick_gpu_ms_mean", C.c_double),
                ("tick_host_ms_mean", C.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class SimConfig(C.Structure):
    _fields_ = [("clients", C.c_int32), ("mean_interarrival_ms", C.c_double), ("min_games", C.c_int32),
                ("max_games", C.c_int32), ("min_side", C.c_int32), ("max_side", C.c_int32),
                ("frac_1v1", C.c_double), ("frac_2v2", C.c_double), ("min_steps", C.c_int32),
                ("max_steps", C.c_int32), ("seconds", C.c_double), ("seed", C.c_uint64),
                ("policy_seed", C.c_uint64), ("budget_bytes", C.c_size_t), ("host_outputs", C.c_int32),
                ("copy_outputs", C.c_int32), ("open_loop", C.c_int32), ("reserved", C.c_int32)]


SERVER_EXPORTS = ("gen_server_create", "gen_server_open", "gen_server_session_layout", "gen_server_step",
                  "gen_server_close", "gen_server_stats_get", "gen_server_destroy", "gen_server_last_error",
                  "gen_server_simulate")


class ServerError(RuntimeError):
    def __init__(self, rc, msg):
        super().__init__(f"({rc}) {msg}")
        self.rc = rc


def _lib():
    lib = load_library()
    if not getattr(lib, "_server_sigs", False):
        vp = C.c_void_p
        sig = {
            "gen_server_create": (C.c_int, [C.POINTER(vp), C.POINTER(GenParams), C.POINTER(ServerConfig)]),
            "gen_server_open": (C.c_int, [vp, C.c_int, vp, vp, vp, vp, C.c_uint64, C.c_int, vp,
                                          C.POINTER(C.c_int32)]),
            "gen_server_session_layout": (C.c_int, [vp, C.c_int, C.POINTER(GenLayoutInfo), vp]),
            "gen_server_step": (C.c_int, [vp, C.c_int, vp, vp, vp, C.POINTER(C.c_double)]),
            "gen_server_close": (C.c_int, [vp, C.c_int]),
            "gen_server_stats_get": (C.c_int, [vp, C.POINTER(ServerStats), C.c_int]),
            "gen_server_destroy": (None, [vp]),
            "gen_server_last_error": (C.c_char_p, []),
            "gen_server_simulate": (C.c_int, [C.POINTER(GenParams), C.POINTER(SimConfig), C.POINTER(ServerStats)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype, f.argtypes = res, args
        lib._server_sigs = True
    return lib


def _check(rc, what):
    if rc != 0:
        raise ServerError(rc, f"{what}: {_lib().gen_server_last_error().decode()}")


def players(mode, n_players):
    return np.where(mode == 0, 2, np.where(mode == 1, 4, n_players)).astype(np.int32)


class SessionBuffers:
    """Host output buffers of one session, in the session's layout."""

    def __init__(self, info: GenLayoutInfo):
        pc, ps, G = int(info.plane_cells), int(info.player_slots), int(info.n_games)
        self.obs_army = np.zeros(pc, np.int16)
        self.obs_owner = np.zeros(pc, np.int8)
        self.obs_terrain = np.zeros(pc, np.int8)
        self.obs_vis = np.zeros(pc, np.uint8)
        self.mask = np.zeros(pc, np.uint8)
        self.reward = np.zeros(ps, np.float32)
        self.scoreboard = np.zeros((ps, 2), np.int32)
        self.done = np.zeros(G, np.uint8)
        self.struct = GenOutputs(*[a.ctypes.data for a in self.arrays()])

    def arrays(self):
        return (self.obs_army, self.obs_owner, self.obs_terrain, self.obs_vis, self.mask, self.reward,
                self.scoreboard, self.done)


class Server:
    def __init__(self, budget_bytes, max_games, max_cells, max_plane_cells, host_outputs=True, policy_seed=2,
                 **params):
        self.lib = _lib()
        self.params = default_params(**params)
        cfg = ServerConfig(int(budget_bytes), int(max_games), int(max_cells), int(max_plane_cells),
                           1 if host_outputs else 0, int(policy_seed))
        h = C.c_void_p()
        _check(self.lib.gen_server_create(C.byref(h), C.byref(self.params), C.byref(cfg)), "gen_server_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.gen_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def open(self, H, W, mode, n_players, game_id_base, wait_ms=0):
        H, W = np.ascontiguousarray(H, np.int32), np.ascontiguousarray(W, np.int32)
        mode, n_players = np.ascontiguousarray(mode, np.int32), np.ascontiguousarray(n_players, np.int32)
        acts = np.zeros(int(players(mode, n_players).sum()), np.int32)
        sid = C.c_int32()
        _check(self.lib.gen_server_open(self.h, int(H.shape[0]), H.ctypes.data, W.ctypes.data, mode.ctypes.data,
                                        n_players.ctypes.data, int(game_id_base), int(wait_ms), acts.ctypes.data,
                                        C.byref(sid)), "gen_server_open")
        return int(sid.value), acts

    def layout(self, session):
        info = GenLayoutInfo()
        _check(self.lib.gen_server_session_layout(self.h, int(session), C.byref(info), None), "session layout")
        return info

    def step(self, session, actions, bufs: SessionBuffers | None, next_actions=None):
        lat = C.c_double()
        nxt = next_actions.ctypes.data if next_actions is not None else None
        _check(self.lib.gen_server_step(self.h, int(session), actions.ctypes.data,
                                        C.byref(bufs.struct) if bufs is not None else None, nxt, C.byref(lat)),
               "gen_server_step")
        return float(lat.value)

    def close_session(self, session):
        _check(self.lib.gen_server_close(self.h, int(session)), "gen_server_close")

    def stats(self, reset=False) -> dict:
        st = ServerStats()
        _check(self.lib.gen_server_stats_get(self.h, C.byref(st), 1 if reset else 0), "stats")
        return st.as_dict()


def simulate(params: dict | None = None, **cfg) -> dict:
    lib = _lib()
    p = default_params(**(params or {}))
    c = SimConfig(**cfg)
    st = ServerStats()
    _check(lib.gen_server_simulate(C.byref(p), C.byref(c), C.byref(st)), "gen_server_simulate")
    return st.as_dict()
