"""Env server: continuous batching of many sessions.  A session's results
are the same alone and in a busy mix, equal the oracle, and sessions are
admitted against the device-memory budget."""
import threading

import numpy as np
import pytest

from oracle import OracleEnv
from paper_2606_23348_gb300.workloads import shapes

pytestmark = pytest.mark.gpu

MB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_23348_gb300.build import build_library
    build_library()


def session_shapes(n, seed, lo=6, hi=16):
    H, W, mode, P = shapes(n, (lo, hi), ((0, 0.4), (1, 0.3), (2, 0.3)), seed=seed)
    P = np.where(mode == 2, np.minimum(P, H * W), P).astype(np.int32)
    return H, W, mode, P


PARAMS = dict(seed=5, min_general_dist=1, n_cities=2, max_turns=25)


def make_server(host_outputs=True, budget=256 * MB):
    from paper_2606_23348_gb300.server import Server
    return Server(budget, max_games=4096, max_cells=4096 * 400, max_plane_cells=4096 * 400 * 8,
                  host_outputs=host_outputs, policy_seed=9, **PARAMS)


def run_session(srv, H, W, mode, P, base, steps):
    from paper_2606_23348_gb300.server import SessionBuffers
    sid, acts = srv.open(H, W, mode, P, base, wait_ms=10000)
    bufs = SessionBuffers(srv.layout(sid))
    hist = []
    for _ in range(steps):
        srv.step(sid, acts, bufs, acts)
        hist.append([a.copy() for a in bufs.arrays()] + [acts.copy()])
    srv.close_session(sid)
    return hist


def test_session_alone_equals_mix_and_oracle():
    H, W, mode, P = session_shapes(12, seed=1)
    base, steps = 1000, 20
    alone = run_session(make_server(), H, W, mode, P, base, steps)

    # the oracle: same games (global ids base + i), same policy seed
    orc = OracleEnv(H, W, mode, P, game_id_base=base, **PARAMS)
    Pn = np.where(mode == 0, 2, np.where(mode == 1, 4, P))
    npad = ((H * W + 15) // 16) * 16
    plane_off = np.concatenate([[0], np.cumsum(Pn * npad)[:-1]])
    slot_off = np.concatenate([[0], np.cumsum(Pn)[:-1]])
    for k in range(steps):
        a = orc.policy(9)
        orc.step(a)
        rec = alone[k]
        for g in range(len(H)):
            s = orc.scalars(g)
            assert rec[7][g] == s["done"], (k, g)
            for p in range(Pn[g]):
                ob = orc.observe(g, p)
                o, n = plane_off[g] + p * npad[g], H[g] * W[g]
                for i, name in enumerate(("army", "owner", "terrain", "vis", "mask")):
                    np.testing.assert_array_equal(rec[i][o:o + n], ob[name], err_msg=f"step {k} game {g} {name}")
                assert rec[5][slot_off[g] + p] == s["reward"][p]
        nxt = orc.policy(9)
        flat = np.concatenate([nxt[g, :Pn[g]] for g in range(len(H))])
        np.testing.assert_array_equal(rec[8], flat, err_msg=f"next actions after step {k}")

    # the mix: other sessions step concurrently from other threads
    srv = make_server()
    stop = threading.Event()
    errors = []

    def other(i):
        try:
            h, w, m, p = session_shapes(20 + 7 * i, seed=100 + i, lo=5, hi=24)
            from paper_2606_23348_gb300.server import SessionBuffers
            while not stop.is_set():
                sid, acts = srv.open(h, w, m, p, 50000 + 1000 * i, wait_ms=10000)
                bufs = SessionBuffers(srv.layout(sid))
                for _ in range(5):
                    srv.step(sid, acts, bufs, acts)
                srv.close_session(sid)
        except Exception as e:  # surfaced below
            errors.append(e)

    th = [threading.Thread(target=other, args=(i,)) for i in range(6)]
    for t in th:
        t.start()
    try:
        mixed = run_session(srv, H, W, mode, P, base, steps)
    finally:
        stop.set()
        for t in th:
            t.join()
    assert not errors, errors
    st = srv.stats()
    assert st["tick_games_mean"] > 12, "the session shared its ticks with others"
    for k in range(steps):
        for x, y in zip(alone[k], mixed[k]):
            np.testing.assert_array_equal(x, y, err_msg=f"step {k}")


def test_device_output_mode_matches_host_mode():
    H, W, mode, P = session_shapes(9, seed=4)
    a = run_session(make_server(host_outputs=True), H, W, mode, P, 77, 8)
    b = run_session(make_server(host_outputs=False), H, W, mode, P, 77, 8)
    for k in range(8):
        for x, y in zip(a[k], b[k]):
            np.testing.assert_array_equal(x, y)


def test_admission_against_budget():
    from paper_2606_23348_gb300.server import ServerError
    H, W, mode, P = session_shapes(40, seed=2, lo=20, hi=20)
    need = int((((H * W + 15) // 16) * 16).sum() * 4 + 40 * 80)
    srv = make_server(budget=int(need * 1.5))
    sid, _ = srv.open(H, W, mode, P, 0)
    with pytest.raises(ServerError):
        srv.open(H, W, mode, P, 100, wait_ms=0)
    got = {}

    def waiter():
        got["sid"] = srv.open(H, W, mode, P, 100, wait_ms=20000)[0]

    t = threading.Thread(target=waiter)
    t.start()
    import time
    time.sleep(0.3)
    assert "sid" not in got
    srv.close_session(sid)
    t.join()
    assert got["sid"] != sid
    st = srv.stats()
    assert st["sessions_waited"] >= 1 and st["sessions_open"] == 1
    assert st["sessions_waited_budget"] >= 1, "the byte budget, not the arenas, held the second session back"
    assert need <= st["peak_bytes_in_use"] <= int(need * 1.5)


def test_simulated_clients_run():
    from paper_2606_23348_gb300.server import simulate
    st = simulate(PARAMS, clients=16, mean_interarrival_ms=1.0, min_games=16, max_games=64, min_side=8,
                  max_side=20, frac_1v1=0.4, frac_2v2=0.3, min_steps=5, max_steps=20, seconds=1.0, seed=3,
                  policy_seed=9, budget_bytes=512 * MB, host_outputs=1, copy_outputs=1)
    assert st["requests"] > 100 and st["frames"] > 0 and st["lat_p99_ms"] >= st["lat_p50_ms"] > 0


def test_open_loop_latency_counts_from_the_scheduled_arrival():
    """Open-loop Poisson clients: every request is timed from its scheduled
    arrival, so the arrival-based percentiles are at least the server-side
    (submission) ones, and an overloaded run (arrivals far faster than the
    steps) queues: its p50 grows well past its service time."""
    from paper_2606_23348_gb300.server import simulate
    base = dict(clients=16, min_games=16, max_games=64, min_side=8, max_side=20, frac_1v1=0.4, frac_2v2=0.3,
                min_steps=5, max_steps=20, seconds=1.0, seed=3, policy_seed=9, budget_bytes=512 * MB,
                host_outputs=1, copy_outputs=1, open_loop=1)
    st = simulate(PARAMS, mean_interarrival_ms=2.0, **base)
    assert st["requests"] > 100 and st["frames"] > 0
    assert st["offered_requests_per_s"] == pytest.approx(16 * 500.0)
    assert st["lat_p99_ms"] >= st["lat_p50_ms"] > 0 and st["service_p99_ms"] >= st["service_p50_ms"] > 0
    assert st["lat_p50_ms"] >= 0.9 * st["service_p50_ms"]
    over = simulate(PARAMS, mean_interarrival_ms=0.001, **base)  # a million requests per second offered
    assert over["lat_p50_ms"] > 5 * over["service_p50_ms"]
