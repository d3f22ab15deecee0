"""Process pool that runs the CPU oracle over disjoint game-id ranges.

TEST INFRASTRUCTURE, like the rest of this directory: used only by the
test-suite and by bench.py's CPU-baseline leg.  Each worker process steps
its own range of games with the oracle (the game id keys the
maps and the policy draws, so ranges are independent) and returns its final
boards or its frame count.  The pool starts with the "spawn" method, so it is
safe after the parent process has initialised CUDA.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time


def _ctx():
    return mp.get_context("spawn")


def _root_on_path():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))  # the repository root
    if root not in sys.path:
        sys.path.insert(0, root)


def _replay(job):
    """Step games [start, start + n) of a workload `frames` times with the
    oracle's benchmark policy; return boards and scalars."""
    _root_on_path()
    import numpy as np

    from oracle import OracleEnv
    name, start, n, seed, policy_seed, frames = job
    from paper_2606_23348_gb300.workloads import workload
    H, W, mode, P, gen, _ = workload(name)
    sl = slice(start, start + n)
    orc = OracleEnv(H[sl], W[sl], mode[sl], P[sl], seed=seed, game_id_base=start, **gen)
    for _ in range(frames):
        orc.step(orc.policy(policy_seed))
    boards = [orc.board(k) for k in range(n)]
    scal = np.array([[orc.scalars(k)[key] for key in ("turn", "frame", "epoch", "alive")] for k in range(n)],
                    np.int64)
    return start, boards, scal


def replay_workload(name: str, games: int, seed: int, policy_seed: int, frames: int, procs: int | None = None,
                    chunk: int = 2048):
    """Oracle boards of the first `games` games of a workload after `frames`
    frames, computed by a spawn pool; list indexed by game."""
    procs = procs or os.cpu_count() or 1
    jobs = [(name, s, min(chunk, games - s), seed, policy_seed, frames) for s in range(0, games, chunk)]
    out = [None] * games
    scal = [None] * games
    with _ctx().Pool(procs) as pool:
        for start, boards, sc in pool.imap_unordered(_replay, jobs):
            for k, b in enumerate(boards):
                out[start + k] = b
                scal[start + k] = sc[k]
    return out, scal


def _throughput(job):
    _root_on_path()
    from oracle import OracleEnv
    from paper_2606_23348_gb300.workloads import workload
    name, start, n, seed, policy_seed, budget_s = job
    H, W, mode, P, gen, _ = workload(name)
    sl = slice(start, start + n)
    orc = OracleEnv(H[sl], W[sl], mode[sl], P[sl], seed=seed, game_id_base=start, **gen)
    frames = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        orc.step(orc.policy(policy_seed))
        frames += 1
    return n * frames, time.perf_counter() - t0


def parallel_throughput(name: str, seed: int, policy_seed: int, budget_s: float, procs: int | None = None,
                        games_per_proc: int = 512):
    """Game-frames/s of `procs` oracle processes on disjoint game ranges, each
    stepping for `budget_s` seconds; returns (value, processes, game-frames)."""
    procs = procs or os.cpu_count() or 1
    jobs = [(name, i * games_per_proc, games_per_proc, seed, policy_seed, budget_s) for i in range(procs)]
    with _ctx().Pool(procs) as pool:
        res = pool.map(_throughput, jobs)
    total = sum(r[0] for r in res)
    return total / max(r[1] for r in res), procs, total
