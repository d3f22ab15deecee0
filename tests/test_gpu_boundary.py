"""The C-ABI's output ownership and saved-state blob, through the library on
cuda:0 and against the oracle byte for byte.

* gen_step / gen_step_policy / gen_observe with a NULL gen_outputs, or with
  some fields NULL, write the environment's own buffers (gen_outputs_get).
* gen_save_state / gen_load_state round-trip one opaque blob: saving, stepping
  ten frames, loading and stepping the same ten frames again gives the same
  bytes, also in a second environment created with another seed.
"""
import numpy as np
import pytest

from gpu_helpers import compare_frame, oracle_actions_flat
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


def _batch(seed=21, G=48):
    H, W, mode, P = shapes(G, (4, 14), ((0, 0.4), (1, 0.3), (2, 0.3)), seed=seed)
    P = np.where(mode == 2, np.minimum(P, H * W), P).astype(np.int32)
    return H, W, mode, P


KW = dict(min_general_dist=1, n_cities=2, max_turns=40)


def test_null_outputs_write_the_environments_own_buffers():
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv, Outputs
    H, W, mode, P = _batch()
    env = GeneralsEnv(H, W, mode, P, seed=5, **KW)
    orc = OracleEnv(H, W, mode, P, seed=5, **KW)
    before = env.device_bytes()
    env.observe(None)
    assert env.device_bytes() > before, "the first NULL-output call allocates the environment's buffers"
    lib_out = env.library_outputs()
    compare_frame(env, lib_out, orc, "observe into own buffers", check_reward=False)
    acts = env.new_actions()
    env.policy(3, acts)
    mine = Outputs(env.layout)
    for f in range(60):
        a_orc = orc.policy(3)
        np.testing.assert_array_equal(acts.cpu().numpy(), oracle_actions_flat(env, a_orc), err_msg=f"frame {f}")
        if f % 3 == 0:
            env.step_policy(acts, None, 3, acts)  # every output to the library's buffers
            got = lib_out
        elif f % 3 == 1:
            # half the fields the caller's, half NULL: each lands where it was asked
            part = Outputs(env.layout)
            part.struct.obs_owner = None
            part.struct.mask = None
            part.struct.done = None
            env.step_policy(acts, part, 3, acts)
            torch.cuda.synchronize()
            for k in ("obs_owner", "mask", "done"):
                setattr(part, k, getattr(lib_out, k))
            got = part
        else:
            env.step_policy(acts, mine, 3, acts)
            got = mine
        orc.step(a_orc)
        compare_frame(env, got, orc, f"frame {f + 1}")
    assert env.read_state()[3][:, 2].max() >= 1, "expected resets within 60 frames (max_turns 40)"


def _record(env, acts, frames, seed=9):
    """Frames of the benchmark policy: every output and the state after each."""
    from paper_2606_23348_gb300.generals import Outputs
    out = Outputs(env.layout)
    rec = []
    for _ in range(frames):
        env.step_policy(acts, out, seed, acts)
        st = env.read_state()
        rec.append([t.cpu().numpy().copy() for t in out.tensors()] + [acts.cpu().numpy().copy()] + list(st))
    return rec


def test_save_step_load_step_gives_identical_bytes():
    from paper_2606_23348_gb300.generals import GeneralsEnv
    H, W, mode, P = _batch(seed=22)
    env = GeneralsEnv(H, W, mode, P, seed=7, **KW)
    orc = OracleEnv(H, W, mode, P, seed=7, **KW)
    acts = env.new_actions()
    env.policy(9, acts)
    for _ in range(25):
        a = orc.policy(9)
        orc.step(a)
    _record(env, acts, 25)
    blob = env.save_state()
    acts0 = acts.clone()
    first = _record(env, acts, 10)
    for _ in range(10):
        orc.step(orc.policy(9))
    compare_frame(env, env.library_outputs(), orc, "after ten frames", check_outputs=False)
    env.load_state(blob)
    acts.copy_(acts0)
    again = _record(env, acts, 10)
    for f, (x, y) in enumerate(zip(first, again)):
        for i, (u, v) in enumerate(zip(x, y)):
            np.testing.assert_array_equal(u, v, err_msg=f"frame {f} array {i}")
    # a second environment of the same shapes but another seed continues the
    # saved games exactly: the blob carries the generator parameters
    other = GeneralsEnv(H, W, mode, P, seed=12345, **KW)
    other.load_state(blob)
    acts.copy_(acts0)
    third = _record(other, acts, 10)
    for f, (x, y) in enumerate(zip(first, third)):
        for i, (u, v) in enumerate(zip(x, y)):
            np.testing.assert_array_equal(u, v, err_msg=f"other env frame {f} array {i}")
    from paper_2606_23348_gb300.generals import Outputs
    out = Outputs(other.layout)
    other.observe(out)
    compare_frame(other, out, orc, "loaded environment vs oracle", check_reward=False)


def test_load_rejects_bad_blobs():
    from paper_2606_23348_gb300.generals import GeneralsEnv, GeneralsError
    H, W, mode, P = _batch(seed=23, G=8)
    env = GeneralsEnv(H, W, mode, P, seed=1, **KW)
    blob = env.save_state()
    before = env.read_state()
    bad = blob.copy()
    bad[len(bad) // 2] ^= 0x40
    with pytest.raises(GeneralsError, match="checksum"):
        env.load_state(bad)
    with pytest.raises(GeneralsError, match="truncated|does not fit"):
        env.load_state(blob[:100])
    bad = blob.copy()
    bad[:8] = 0
    with pytest.raises(GeneralsError, match="not a saved"):
        env.load_state(bad)
    H2 = H.copy()
    H2[0] = H2[0] + 1 if H2[0] < 14 else H2[0] - 1
    env2 = GeneralsEnv(H2, W, mode, P, seed=1, **KW)
    with pytest.raises(GeneralsError):
        env2.load_state(blob)
    after = env.read_state()
    for x, y in zip(before, after):
        np.testing.assert_array_equal(x, y)  # a refused blob changes nothing


def test_misaligned_outputs_are_refused_on_the_host():
    """Output planes are written 16 bytes at a time and the reward and
    scoreboard one 4-byte word at a time: pointers that break either are
    refused before any launch, and the environment stays usable."""
    import torch

    from paper_2606_23348_gb300.generals import GeneralsEnv, GeneralsError
    H, W, mode, P = _batch(seed=24, G=8)
    env = GeneralsEnv(H, W, mode, P, seed=1, **KW)
    acts = env.new_actions()
    spare = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    for field, offset in (("obs_army", 8), ("mask", 4), ("reward", 2), ("scoreboard", 1)):
        out = env.new_outputs()
        setattr(out.struct, field, spare.data_ptr() + offset)
        with pytest.raises(GeneralsError, match="aligned"):
            env.step(acts, out)
    import ctypes as C
    out = env.new_outputs()
    odd = C.c_void_p(acts.data_ptr() + 2)
    assert env.lib.gen_step(env.h, odd, C.byref(out.struct), None) != 0  # actions read as int32
    assert env.lib.gen_policy(env.h, 1, odd, None) != 0
    env.step(acts, out)  # still usable
    torch.cuda.synchronize()
    assert env.read_state()[3][:, 7].max() == 0
