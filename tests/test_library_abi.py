"""The C-ABI library loads and exports every entry point include/generals.h
declares; host-side argument checks reject bad input before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2606_23348_gb300.generals as gen
from paper_2606_23348_gb300.build import build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "generals.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gen_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build_library()
    return gen.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared but not exported"
    from paper_2606_23348_gb300.server import SERVER_EXPORTS
    assert set(names) == set(gen.EXPORTS) | set(SERVER_EXPORTS)


def test_default_params_host_only(lib):
    p = gen.default_params()
    assert p.mountain_thresh == 858993459 and p.city_army_min == 40 and p.city_army_max == 50
    assert p.auto_reset == 1 and p.max_turns == 0 and p.min_general_dist == 0


@pytest.mark.parametrize("H,W,mode,P", [(65, 10, 0, 2), (0, 5, 0, 2), (1, 1, 0, 2), (2, 2, 3, 2), (2, 3, 2, 9),
                                        (2, 3, 2, 1), (1, 3, 1, 4)])
def test_create_rejects_bad_shapes(lib, H, W, mode, P):
    p = gen.default_params()
    h = C.c_void_p()
    arr = lambda v: np.array([v], np.int32)
    Hs, Ws, Ms, Ps = arr(H), arr(W), arr(mode), arr(P)
    rc = lib.gen_create_ex(C.byref(h), C.byref(p), 1, Hs.ctypes.data, Ws.ctypes.data, Ms.ctypes.data,
                           Ps.ctypes.data)
    assert rc == -1 and not h.value
    assert lib.gen_last_error().decode()


def test_create_rejects_bad_params(lib):
    h = C.c_void_p()
    one = np.array([10], np.int32)
    zero = np.array([0], np.int32)
    for kw in (dict(city_army_min=50, city_army_max=40), dict(max_turns=-1),
               dict(n_cities=-1, city_per_mille=2000)):
        p = gen.default_params(**kw)
        assert lib.gen_create_ex(C.byref(h), C.byref(p), 1, one.ctypes.data, one.ctypes.data, zero.ctypes.data,
                                 zero.ctypes.data) == -1
    p = gen.default_params()
    assert lib.gen_create_ex(C.byref(h), C.byref(p), 0, one.ctypes.data, one.ctypes.data, zero.ctypes.data,
                             zero.ctypes.data) == -1


def test_null_env_calls_fail_cleanly(lib):
    out = gen.GenOutputs()
    assert lib.gen_step(None, None, C.byref(out), None) == -1
    assert lib.gen_policy(None, 0, None, None) == -1
    assert lib.gen_set_launch(None, 8) == -1
    assert lib.gen_copy_peak(0, 1, None) == -1


def test_null_handles_of_the_form_switches_fail_cleanly(lib):
    """The launch-form switches refuse a NULL handle with GEN_ERR_BAD_ARG and a
    message, on the host, before any CUDA call."""
    for call in (lambda: lib.gen_set_lane_groups(None, 0), lambda: lib.gen_set_sample_form(None, 0),
                 lambda: lib.gen_features_set_form(None, 0), lambda: lib.gen_set_spawn_range(None, 0, 0)):
        assert call() == -1
        assert lib.gen_last_error().decode()


def test_boundary_additions_refuse_null_handles(lib):
    """The saved-state blob, the environment's own outputs and the byte count
    refuse NULL arguments on the host, before any CUDA call."""
    used = C.c_size_t()
    out = gen.GenOutputs()
    buf = (C.c_ubyte * 256)()
    for call in (lambda: lib.gen_save_state(None, None, 0, C.byref(used), None),
                 lambda: lib.gen_load_state(None, buf, 256, None),
                 lambda: lib.gen_outputs_get(None, C.byref(out)),
                 lambda: lib.gen_device_bytes(None, C.byref(used))):
        assert call() == -1
        assert lib.gen_last_error().decode()
