"""The N-rank path on CPU (gloo, world size 2): ranks step disjoint game-id
ranges with no exchange; together they reproduce one process stepping every
game (boards, scalars, feature tensors, temporal tokens and sampled actions,
all keyed by the global game id), and the benchmark's reductions over ranks
(max time, summed frames) behave as stated.  The oracle stands in for each
rank's GPU here."""
import hashlib
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from oracle import OracleEnv
from paper_2606_23348_gb300.workloads import shapes, shard

G_PER_RANK = 12
FRAMES = 30
KW = dict(seed=4, min_general_dist=1, n_cities=2, max_turns=20)


def digest(env, g):
    h = hashlib.sha1()
    for a in env.board(g):
        h.update(a.tobytes())
    s = env.scalars(g)
    h.update(repr((s["turn"], s["epoch"], s["alive"], s["frame"])).encode())
    return h.hexdigest()


def run_games(base, H, W, mode, P):
    """Boards, scalars, the feature tensor with temporal tokens, and an action
    sampled from logits seeded by the global game id, per game."""
    from oracle.orc import OracleFeatures
    env = OracleEnv(H, W, mode, P, game_id_base=base, **KW)
    feats = OracleFeatures(env, hist=3, window=8)
    for _ in range(FRAMES):
        env.step(env.policy(3))
        f = feats.build()
    logits = [np.random.default_rng(base + g).normal(0, 2, (int(env.P[g]), 9 * int(env.N[g]))).astype(np.float32)
              for g in range(env.G)]
    acts, _ = env.sample_actions(logits, 17)
    out = []
    for g in range(env.G):
        h = hashlib.sha1(digest(env, g).encode())
        h.update(f[g].tobytes())
        h.update(feats.series[g].tobytes())
        h.update(acts[g].tobytes())
        out.append(h.hexdigest())
    return out


def rank_main(rank, world, port, H, W, mode, P, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo = rank * G_PER_RANK
    mine = run_games(shard(G_PER_RANK, rank), H[lo:lo + G_PER_RANK], W[lo:lo + G_PER_RANK],
                     mode[lo:lo + G_PER_RANK], P[lo:lo + G_PER_RANK])
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    import bench
    t = bench.max_over_ranks(float(rank + 1), world)
    n = bench.sum_over_ranks(float(G_PER_RANK), world)
    if rank == 0:
        q.put((sum(gathered, []), t, n))
    dist.barrier()
    dist.destroy_process_group()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_equal_one_process():
    world = 2
    H, W, mode, P = shapes(world * G_PER_RANK, (4, 10), ((0, 0.5), (1, 0.25), (2, 0.25)), seed=6)
    P = np.where(mode == 2, np.minimum(P, H * W), P).astype(np.int32)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, H, W, mode, P, q)) for r in range(world)]
    for p in procs:
        p.start()
    got, t, n = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == run_games(0, H, W, mode, P)
    assert t == 2.0 and n == world * G_PER_RANK


def test_bench_starts_its_own_ranks():
    """`bench.py --gpus 2` started without a launcher runs itself as two ranks
    (torch.distributed.run, gloo on a host without a GPU, rendezvous on
    127.0.0.1) and prints one line from rank 0.  The reference arm needs no
    GPU, so the whole N-rank path of the bench runs here."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    env.pop("WORLD_SIZE", None)
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--impl", "reference",
                        "--steps", "2", "--warmup", "3"], capture_output=True, text=True, timeout=300, env=env,
                       cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
