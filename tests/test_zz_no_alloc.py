"""gen_step_host_static: the host-buffer step for callers that cannot
allocate device memory (an actor whose device memory is already handed to a
fixed-size pool, or a real-time loop that must not take cudaMalloc's implicit
synchronisation or risk running out of memory mid-rollout).  It stages
through the library's static device array and must return exactly what
gen_step_host returns, call after call.  This file is collected last."""
import numpy as np
import pytest

from paper_2606_23348_gb300.workloads import shapes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_23348_gb300.build import build_library
    build_library()


def _env():
    from paper_2606_23348_gb300.generals import GeneralsEnv
    H, W, mode, P = shapes(96, (6, 24), ((0, 0.5), (1, 0.25), (2, 0.25)), seed=13)
    return GeneralsEnv(H, W, mode, P, seed=13, min_general_dist=1, n_cities=3, max_turns=30)


def test_static_stage_matches_host_step_on_consecutive_calls():
    import torch
    from paper_2606_23348_gb300.generals import Outputs
    env_a, env_b = _env(), _env()  # identical batches: same shapes, seeds and parameters
    out_a = Outputs(env_a.layout, pin_host=True)
    out_b = Outputs(env_b.layout, pin_host=True)
    d_act = env_a.new_actions()
    env_a.policy(17, d_act)
    act_a = d_act.cpu().pin_memory()
    act_b = act_a.clone().pin_memory()
    nxt_a = torch.empty_like(act_a).pin_memory()
    nxt_b = torch.empty_like(act_b).pin_memory()
    held = env_b.device_bytes()  # env_b only ever takes the static path
    for call in range(2):
        env_a.step_host(act_a, out_a, 17, nxt_a)
        env_b.step_host_static(act_b, out_b, 17, nxt_b)
        for x, y in zip(out_a.tensors(), out_b.tensors()):
            np.testing.assert_array_equal(x.numpy(), y.numpy(), err_msg=f"call {call}")
        np.testing.assert_array_equal(nxt_a.numpy(), nxt_b.numpy(), err_msg=f"call {call}")
        act_a.copy_(nxt_a)
        act_b.copy_(nxt_b)
        assert env_b.device_bytes() == held, "the static entry point allocated device memory"


def test_static_stage_rejects_batches_beyond_its_size():
    import torch
    from paper_2606_23348_gb300.generals import GeneralsEnv, GeneralsError, Outputs
    env = GeneralsEnv(64, 64, 0, 2, batch=700, seed=2)  # 5.7 M plane cells: more than 32 MiB of staging
    out = Outputs(env.layout, pin_host=True)
    act = torch.zeros(int(env.layout.player_slots), dtype=torch.int32).pin_memory()
    with pytest.raises(GeneralsError, match="at most"):
        env.step_host_static(act, out)
