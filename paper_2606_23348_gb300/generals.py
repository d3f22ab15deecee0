"""Python binding of libgenerals (include/generals.h) — argument marshalling only.

Every step of the environment runs in the library's CUDA kernels; this module
allocates torch tensors for the outputs, passes their device pointers and
the current CUDA stream through ctypes, and raises when a call fails.  There
is no CPU fallback: without the compiled library and a GPU nothing here runs.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libgenerals.so")
_lock = threading.Lock()
_lib = None

GEN_MAX_PLAYERS = 8


class GenParams(C.Structure):
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


class GenOutputs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in
                ("obs_army", "obs_owner", "obs_terrain", "obs_vis", "mask", "reward", "scoreboard", "done")]


class GenLayoutInfo(C.Structure):
    _fields_ = [
        ("n_games", C.c_int32),
        ("player_slots", C.c_int32),
        ("plane_cells", C.c_int64),
        ("state_cells", C.c_int64),
        ("max_players", C.c_int32),
        ("max_cells", C.c_int32),
    ]


EXPORTS = ("gen_default_params", "gen_create", "gen_create_ex", "gen_layout", "gen_reset", "gen_observe",
           "gen_step", "gen_step_policy", "gen_policy", "gen_rollout", "gen_step_host", "gen_read_state",
           "gen_write_state", "gen_set_launch", "gen_autotune", "gen_copy_peak", "gen_last_error", "gen_destroy",
           "gen_step_host_static", "gen_set_spawn_range", "gen_features_create", "gen_features_layout",
           "gen_features_build", "gen_features_destroy", "gen_features_create_ex", "gen_features_series_layout",
           "gen_features_build_ex", "gen_features_set_form", "gen_sample_actions", "gen_set_sample_form",
           "gen_set_lane_groups", "gen_outputs_get", "gen_device_bytes", "gen_save_state", "gen_load_state",
           "gen_set_batch_form", "gen_features_autotune")

ROLLOUT_RESIDENT, ROLLOUT_GRAPH, ROLLOUT_LAUNCHES, ROLLOUT_AUTO = 0, 1, 2, 3


def load_library(path: str = LIB_PATH):
    """Load libgenerals.so; raise if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libgenerals.so is not built ({path}); run __graft_entry__.build() or "
                               "python -m paper_2606_23348_gb300.build")
        lib = C.CDLL(path)
        vp, i32, u64 = C.c_void_p, C.c_int32, C.c_uint64
        sig = {
            "gen_default_params": (C.c_int, [C.POINTER(GenParams)]),
            "gen_create": (C.c_int, [C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.c_int, u64]),
            "gen_create_ex": (C.c_int, [C.POINTER(vp), C.POINTER(GenParams), C.c_int, vp, vp, vp, vp]),
            "gen_layout": (C.c_int, [vp, C.POINTER(GenLayoutInfo), vp, vp, vp]),
            "gen_reset": (C.c_int, [vp, vp, C.c_int, C.POINTER(GenOutputs), vp]),
            "gen_observe": (C.c_int, [vp, C.POINTER(GenOutputs), vp]),
            "gen_step": (C.c_int, [vp, vp, C.POINTER(GenOutputs), vp]),
            "gen_step_policy": (C.c_int, [vp, vp, C.POINTER(GenOutputs), u64, vp, vp]),
            "gen_policy": (C.c_int, [vp, u64, vp, vp]),
            "gen_rollout": (C.c_int, [vp, C.c_int, u64, vp, C.POINTER(GenOutputs), vp, C.c_int, vp]),
            "gen_autotune": (C.c_int, [vp, C.c_int, C.c_char_p, C.c_size_t]),
            "gen_step_host": (C.c_int, [vp, vp, C.POINTER(GenOutputs), u64, vp, vp]),
            "gen_step_host_static": (C.c_int, [vp, vp, C.POINTER(GenOutputs), u64, vp, vp]),
            "gen_read_state": (C.c_int, [vp, vp, vp, vp, vp, vp]),
            "gen_write_state": (C.c_int, [vp, vp, vp, vp, vp, vp]),
            "gen_set_launch": (C.c_int, [vp, C.c_int]),
            "gen_set_spawn_range": (C.c_int, [vp, C.c_int, C.c_int]),
            "gen_copy_peak": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(C.c_double)]),
            "gen_features_create": (C.c_int, [C.POINTER(vp), vp, C.c_int]),
            "gen_features_layout": (C.c_int, [vp, C.POINTER(i32), C.POINTER(C.c_int64)]),
            "gen_features_build": (C.c_int, [vp, vp, vp]),
            "gen_features_destroy": (None, [vp]),
            "gen_features_create_ex": (C.c_int, [C.POINTER(vp), vp, C.c_int, C.c_int]),
            "gen_features_series_layout": (C.c_int, [vp, C.POINTER(i32), C.POINTER(C.c_int64)]),
            "gen_features_build_ex": (C.c_int, [vp, vp, vp, vp]),
            "gen_features_set_form": (C.c_int, [vp, C.c_int]),
            "gen_sample_actions": (C.c_int, [vp, vp, u64, vp, vp, vp]),
            "gen_set_sample_form": (C.c_int, [vp, C.c_int]),
            "gen_set_lane_groups": (C.c_int, [vp, C.c_int]),
            "gen_outputs_get": (C.c_int, [vp, C.POINTER(GenOutputs)]),
            "gen_set_batch_form": (C.c_int, [vp, C.c_int]),
            "gen_features_autotune": (C.c_int, [vp, vp, C.c_int, C.POINTER(i32)]),
            "gen_device_bytes": (C.c_int, [vp, C.POINTER(C.c_size_t)]),
            "gen_save_state": (C.c_int, [vp, vp, C.c_size_t, C.POINTER(C.c_size_t), vp]),
            "gen_load_state": (C.c_int, [vp, vp, C.c_size_t, vp]),
            "gen_last_error": (C.c_char_p, []),
            "gen_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


class GeneralsError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise GeneralsError(f"{what} failed ({rc}): {load_library().gen_last_error().decode()}")


def default_params(**kw) -> GenParams:
    p = GenParams()
    _check(load_library().gen_default_params(C.byref(p)), "gen_default_params")
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def copy_peak_gbps(nbytes: int = 1 << 30, reps: int = 10) -> float:
    """HBM copy bandwidth (read + write bytes) measured by the library's own copy kernel."""
    out = C.c_double()
    _check(load_library().gen_copy_peak(nbytes, reps, C.byref(out)), "gen_copy_peak")
    return float(out.value)


def _cur_stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Outputs:
    """Device output tensors of one environment (torch, on cuda); `frames`
    consecutive frames for rollouts."""

    def __init__(self, layout: GenLayoutInfo, device="cuda", pin_host: bool = False, frames: int = 1):
        import torch
        pc, ps, G = (int(layout.plane_cells) * frames, int(layout.player_slots) * frames,
                     int(layout.n_games) * frames)
        kw = dict(device=device) if not pin_host else dict(pin_memory=True)
        self.obs_army = torch.empty(pc, dtype=torch.int16, **kw)
        self.obs_owner = torch.empty(pc, dtype=torch.int8, **kw)
        self.obs_terrain = torch.empty(pc, dtype=torch.int8, **kw)
        self.obs_vis = torch.empty(pc, dtype=torch.uint8, **kw)
        self.mask = torch.empty(pc, dtype=torch.uint8, **kw)
        self.reward = torch.empty(ps, dtype=torch.float32, **kw)
        self.scoreboard = torch.empty((ps, 2), dtype=torch.int32, **kw)
        self.done = torch.empty(G, dtype=torch.uint8, **kw)
        self.struct = GenOutputs(*[t.data_ptr() for t in self.tensors()])

    def tensors(self):
        return (self.obs_army, self.obs_owner, self.obs_terrain, self.obs_vis, self.mask, self.reward,
                self.scoreboard, self.done)

    def nbytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in self.tensors())


class _DevicePtr:
    """A device buffer the library owns, seen by torch through the CUDA array
    interface (zero copy)."""

    def __init__(self, ptr: int, n: int, typestr: str, shape=None):
        self.__cuda_array_interface__ = {"shape": shape or (n,), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class LibraryOutputs(Outputs):
    """Torch views of an environment's own output buffers (gen_outputs_get):
    what gen_step writes for NULL output fields, valid until the environment
    is destroyed."""

    def __init__(self, env: "GeneralsEnv"):  # noqa: super() not called: the library owns the memory
        import torch
        st = GenOutputs()
        _check(env.lib.gen_outputs_get(env.h, C.byref(st)), "gen_outputs_get")
        pc, ps, G = int(env.layout.plane_cells), int(env.layout.player_slots), int(env.layout.n_games)
        view = lambda ptr, n, t, shape=None: torch.as_tensor(_DevicePtr(ptr, n, t, shape), device="cuda")
        self.obs_army = view(st.obs_army, pc, "<i2")
        self.obs_owner = view(st.obs_owner, pc, "|i1")
        self.obs_terrain = view(st.obs_terrain, pc, "|i1")
        self.obs_vis = view(st.obs_vis, pc, "|u1")
        self.mask = view(st.mask, pc, "|u1")
        self.reward = view(st.reward, ps, "<f4")
        self.scoreboard = view(st.scoreboard, ps, "<i4", (ps, 2))
        self.done = view(st.done, G, "|u1")
        self.struct = st
        self.env = env  # keeps the environment (and its buffers) alive


class GeneralsEnv:
    """A batch of games held on the GPU by libgenerals.

    ``H``, ``W``, ``mode`` and ``n_players`` are per-game sequences (ragged
    batches allowed) or scalars with ``batch``.
    """

    def __init__(self, H, W, mode=0, n_players=8, batch=None, **params):
        lib = load_library()
        if batch is not None:
            H, W = np.full(batch, H), np.full(batch, W)
            mode, n_players = np.full(batch, mode), np.full(batch, n_players)
        self.H = np.ascontiguousarray(H, np.int32)
        self.W = np.ascontiguousarray(W, np.int32)
        self.mode = np.ascontiguousarray(np.broadcast_to(mode, self.H.shape), np.int32)
        self.n_players = np.ascontiguousarray(np.broadcast_to(n_players, self.H.shape), np.int32)
        self.params = default_params(**params)
        h = C.c_void_p()
        _check(lib.gen_create_ex(C.byref(h), C.byref(self.params), int(self.H.shape[0]),
                                 self.H.ctypes.data, self.W.ctypes.data, self.mode.ctypes.data,
                                 self.n_players.ctypes.data), "gen_create_ex")
        self.h = h
        self.lib = lib
        info = GenLayoutInfo()
        G = int(self.H.shape[0])
        self.plane_off = np.zeros(G, np.int64)
        self.player_off = np.zeros(G, np.int32)
        self.npad = np.zeros(G, np.int32)
        _check(lib.gen_layout(h, C.byref(info), self.plane_off.ctypes.data, self.player_off.ctypes.data,
                              self.npad.ctypes.data), "gen_layout")
        self.layout = info
        self.G = G
        self.P = np.where(self.mode == 0, 2, np.where(self.mode == 1, 4, self.n_players)).astype(np.int32)
        self.N = (self.H * self.W).astype(np.int64)
        self.state_off = np.concatenate([[0], np.cumsum(self.npad)[:-1]]).astype(np.int64)

    def close(self):
        if getattr(self, "h", None):
            self.lib.gen_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- buffers --------------------------------------------------------
    def new_outputs(self, frames: int = 1) -> Outputs:
        return Outputs(self.layout, frames=frames)

    def new_actions(self):
        import torch
        return torch.zeros(int(self.layout.player_slots), dtype=torch.int32, device="cuda")

    # ---- calls ----------------------------------------------------------
    def observe(self, out: Outputs | None = None, stream=None):
        ref = C.byref(out.struct) if out is not None else None
        _check(self.lib.gen_observe(self.h, ref, stream or _cur_stream()), "gen_observe")

    def reset(self, out: Outputs, game_ids=None, stream=None):
        if game_ids is None:
            _check(self.lib.gen_reset(self.h, None, 0, C.byref(out.struct), stream or _cur_stream()), "gen_reset")
        else:
            _check(self.lib.gen_reset(self.h, C.c_void_p(game_ids.data_ptr()), int(game_ids.numel()),
                                      C.byref(out.struct), stream or _cur_stream()), "gen_reset")

    def step(self, actions, out: Outputs | None = None, stream=None):
        """One turn of every game; out=None writes the environment's own
        buffers (library_outputs())."""
        ref = C.byref(out.struct) if out is not None else None
        _check(self.lib.gen_step(self.h, C.c_void_p(actions.data_ptr()), ref, stream or _cur_stream()), "gen_step")

    def library_outputs(self) -> LibraryOutputs:
        """Torch views of the environment's own output buffers."""
        return LibraryOutputs(self)

    def device_bytes(self) -> int:
        n = C.c_size_t()
        _check(self.lib.gen_device_bytes(self.h, C.byref(n)), "gen_device_bytes")
        return int(n.value)

    def save_state(self) -> np.ndarray:
        """Everything that determines later frames, as one opaque host blob (uint8)."""
        need = C.c_size_t()
        _check(self.lib.gen_save_state(self.h, None, 0, C.byref(need), _cur_stream()), "gen_save_state")
        buf = np.empty(int(need.value), np.uint8)
        used = C.c_size_t()
        _check(self.lib.gen_save_state(self.h, buf.ctypes.data, buf.nbytes, C.byref(used), _cur_stream()),
               "gen_save_state")
        return buf[:int(used.value)]

    def load_state(self, blob):
        blob = np.ascontiguousarray(blob, np.uint8)
        _check(self.lib.gen_load_state(self.h, blob.ctypes.data, blob.nbytes, _cur_stream()), "gen_load_state")

    def step_policy(self, actions, out: Outputs | None, policy_seed: int, next_actions, stream=None):
        ref = C.byref(out.struct) if out is not None else None
        _check(self.lib.gen_step_policy(self.h, C.c_void_p(actions.data_ptr()), ref,
                                        int(policy_seed), C.c_void_p(next_actions.data_ptr()),
                                        stream or _cur_stream()), "gen_step_policy")

    def policy(self, policy_seed: int, actions, stream=None):
        _check(self.lib.gen_policy(self.h, int(policy_seed), C.c_void_p(actions.data_ptr()),
                                   stream or _cur_stream()), "gen_policy")

    def rollout(self, K: int, policy_seed: int, actions, out: Outputs, action_log=None, form: int = 0,
                stream=None):
        log = C.c_void_p(action_log.data_ptr()) if action_log is not None else None
        _check(self.lib.gen_rollout(self.h, int(K), int(policy_seed), C.c_void_p(actions.data_ptr()),
                                    C.byref(out.struct), log, int(form), stream or _cur_stream()), "gen_rollout")

    def autotune(self, steps: int = 5) -> str:
        buf = C.create_string_buffer(4096)
        _check(self.lib.gen_autotune(self.h, int(steps), buf, 4096), "gen_autotune")
        return buf.value.decode()

    def step_host(self, h_actions, h_out: Outputs, policy_seed: int = 0, h_next_actions=None, stream=None):
        """Host-buffer step: h_actions, h_out (and h_next_actions) are CPU (pinned) tensors."""
        nxt = C.c_void_p(h_next_actions.data_ptr()) if h_next_actions is not None else None
        _check(self.lib.gen_step_host(self.h, C.c_void_p(h_actions.data_ptr()), C.byref(h_out.struct),
                                      int(policy_seed), nxt, stream or _cur_stream()), "gen_step_host")

    def step_host_static(self, h_actions, h_out: Outputs, policy_seed: int = 0, h_next_actions=None,
                         stream=None):
        """step_host staged through the library's static device array (no device allocation)."""
        nxt = C.c_void_p(h_next_actions.data_ptr()) if h_next_actions is not None else None
        _check(self.lib.gen_step_host_static(self.h, C.c_void_p(h_actions.data_ptr()), C.byref(h_out.struct),
                                             int(policy_seed), nxt, stream or _cur_stream()),
               "gen_step_host_static")

    def set_spawn_range(self, min_dist: int, max_dist: int):
        _check(self.lib.gen_set_spawn_range(self.h, int(min_dist), int(max_dist)), "gen_set_spawn_range")

    def new_logits(self):
        """Zero logits: 9 float32 per cell of every player plane."""
        import torch
        return torch.zeros(int(self.layout.plane_cells) * 9, dtype=torch.float32, device="cuda")

    LANES_AUTO, LANES_WARP, LANES_NARROW = 0, 1, 2

    def set_lane_groups(self, mode: int):
        """Games per warp in the step kernels: LANES_WARP (one), LANES_NARROW
        (two, four in rollouts, wherever the games allow) or LANES_AUTO (by
        batch size)."""
        _check(self.lib.gen_set_lane_groups(self.h, int(mode)), "gen_set_lane_groups")

    BATCH_AUTO, BATCH_BUCKETS, BATCH_WORKLIST = 0, 1, 2

    def set_batch_form(self, form: int):
        """How a batch of several size buckets launches: BATCH_BUCKETS (one
        launch per bucket), BATCH_WORKLIST (one persistent work-list launch)
        or BATCH_AUTO (the work list for batches of more than four buckets)."""
        _check(self.lib.gen_set_batch_form(self.h, int(form)), "gen_set_batch_form")

    def set_sample_form(self, form: int):
        """How sample_actions spreads a game over the GPU: 1 one warp per
        game, 2 one CTA per game with a warp per player, 3 one CTA per player
        with a thread per (own cell, entry), 0 the default (by batch size)."""
        _check(self.lib.gen_set_sample_form(self.h, int(form)), "gen_set_sample_form")

    def sample_actions(self, logits, seed: int, actions=None, mask9=None):
        """Draw one action per player from `logits` (9 per plane cell) into
        `actions` (allocated when None); `mask9` (uint8, 9 per plane cell)
        receives the expanded legal mask when given."""
        if actions is None:
            actions = self.new_actions()
        mp = C.c_void_p(mask9.data_ptr()) if mask9 is not None else None
        _check(self.lib.gen_sample_actions(self.h, C.c_void_p(logits.data_ptr()), int(seed),
                                           C.c_void_p(actions.data_ptr()), mp, _cur_stream()), "gen_sample_actions")
        return actions

    def expand_mask(self, mask9=None):
        """The expanded H x W x 9 legal mask of every player (uint8, 9 per plane cell)."""
        import torch
        if mask9 is None:
            mask9 = torch.empty(int(self.layout.plane_cells) * 9, dtype=torch.uint8, device="cuda")
        _check(self.lib.gen_sample_actions(self.h, None, 0, None, C.c_void_p(mask9.data_ptr()), _cur_stream()),
               "gen_sample_actions")
        return mask9

    def features(self, hist: int = 7, window: int = 0) -> "Features":
        """Feature-tensor builder over this environment (App. A); window > 0
        adds the temporal tokens (opponents' army and land, newest first)."""
        return Features(self, hist, window)

    def set_launch(self, warps_per_cta: int):
        _check(self.lib.gen_set_launch(self.h, int(warps_per_cta)), "gen_set_launch")

    def read_state(self):
        n = int(self.layout.state_cells)
        army = np.zeros(n, np.int16)
        owner = np.zeros(n, np.int8)
        terrain = np.zeros(n, np.int8)
        scal = np.zeros((self.G, 8), np.uint32)
        _check(self.lib.gen_read_state(self.h, army.ctypes.data, owner.ctypes.data, terrain.ctypes.data,
                                       scal.ctypes.data, _cur_stream()), "gen_read_state")
        return army, owner, terrain, scal

    def write_state(self, army, owner, terrain, scal):
        army = np.ascontiguousarray(army, np.int16)
        owner = np.ascontiguousarray(owner, np.int8)
        terrain = np.ascontiguousarray(terrain, np.int8)
        scal = np.ascontiguousarray(scal, np.uint32)
        _check(self.lib.gen_write_state(self.h, army.ctypes.data, owner.ctypes.data, terrain.ctypes.data,
                                        scal.ctypes.data, _cur_stream()), "gen_write_state")

    # ---- views ----------------------------------------------------------
    def board(self, state, g: int):
        """(army, owner, terrain) of game g from a read_state() tuple, padding removed."""
        o, n = int(self.state_off[g]), int(self.N[g])
        return state[0][o:o + n], state[1][o:o + n], state[2][o:o + n]

    def plane(self, t, g: int, p: int):
        """Player p's plane of game g from a flat per-player output tensor (padding removed)."""
        o = int(self.plane_off[g]) + p * int(self.npad[g])
        return t[o:o + int(self.N[g])]


class Features:
    """The 24 + 2 * hist channel feature tensor of every player (gen_features_*).

    ``build()`` folds the current frame into the per-player memory and
    returns a float32 device tensor of ``n_floats`` (a uniform batch views as
    [G][P][C][H*W]); call it after every step.
    """

    def __init__(self, env: GeneralsEnv, hist: int = 7, window: int = 0):
        self.env = env
        self.lib = env.lib
        h = C.c_void_p()
        _check(self.lib.gen_features_create_ex(C.byref(h), env.h, int(hist), int(window)), "gen_features_create_ex")
        self.h = h
        ch, n = C.c_int32(), C.c_int64()
        _check(self.lib.gen_features_layout(h, C.byref(ch), C.byref(n)), "gen_features_layout")
        self.channels, self.n_floats, self.hist = int(ch.value), int(n.value), int(hist)
        w, ns = C.c_int32(), C.c_int64()
        _check(self.lib.gen_features_series_layout(h, C.byref(w), C.byref(ns)), "gen_features_series_layout")
        self.window, self.n_series = int(w.value), int(ns.value)

    def new_output(self):
        import torch
        return torch.empty(self.n_floats, dtype=torch.float32, device="cuda")

    def new_series(self):
        import torch
        return torch.empty(self.n_series, dtype=torch.int32, device="cuda")

    def build(self, out=None, series=None):
        """Features into `out` (allocated when None); with `series` (a tensor
        of n_series int32) the temporal tokens too."""
        if self.env.h is None:
            raise GeneralsError("the environment of this feature builder is closed")
        if out is None:
            out = self.new_output()
        assert out.numel() >= self.n_floats and out.dtype.itemsize == 4 and out.is_cuda
        sp = None
        if series is not None:
            assert series.numel() >= self.n_series and series.dtype.itemsize == 4 and series.is_cuda
            sp = C.c_void_p(series.data_ptr())
        _check(self.lib.gen_features_build_ex(self.h, C.c_void_p(out.data_ptr()), sp, _cur_stream()),
               "gen_features_build_ex")
        return out

    FORM_AUTO, FORM_WARP, FORM_CTA = 0, 1, 2

    def autotune(self, out, steps: int = 5) -> int:
        """Time both forms building into `out` and keep the faster; returns it."""
        f = C.c_int32()
        _check(self.lib.gen_features_autotune(self.h, C.c_void_p(out.data_ptr()), int(steps), C.byref(f)),
               "gen_features_autotune")
        return int(f.value)

    def set_form(self, form: int):
        """Spread of a game over the GPU: FORM_WARP (one warp per game),
        FORM_CTA (one CTA per game and player, for small batches) or
        FORM_AUTO."""
        _check(self.lib.gen_features_set_form(self.h, int(form)), "gen_features_set_form")

    def player_series(self, series, g: int, p: int):
        """[T][2] (army, land) view of game g, player p inside a series output."""
        s = int(self.env.player_off[g]) + p
        return series[s * 2 * self.window:(s + 1) * 2 * self.window].view(self.window, 2)

    def player_view(self, out, g: int, p: int):
        """[C][H_g * W_g] view of game g, player p inside a build() output."""
        npad = int(self.env.npad[g])
        q = int(self.env.plane_off[g]) + p * npad
        n = int(self.env.H[g]) * int(self.env.W[g])
        C = self.channels
        return out[q * C:q * C + C * npad].view(C, npad)[:, :n]

    def close(self):
        if getattr(self, "h", None):
            self.lib.gen_features_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
