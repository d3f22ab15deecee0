"""Throughput of the batched Generals.io environment step on GB300.

One benchmark step = one frame of every game of the workload: the fused
step kernel (moves, combat, capture, growth, termination, reward, auto-reset,
fog, observations, mask, scoreboard) plus the benchmark random-legal policy
that produces the next frame's actions, in one launch.  Default workload:
65,536 1v1 games on 24x24 boards (20% mountains, 12 castles of 40-50),
auto-reset on, synthetic and seeded.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank steps its own
games (global ids offset by rank) with no collective on the data path.
``--impl reference`` times the CPU oracle (the only other implementation of
these rules) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "1v1-65536x24x24"
STEP_PREROLL = 256  # frames of the benchmark policy before the default workload's warm-up and timed steps
METRIC = "frames/s per GB300 (bit-exact vs oracle)"
UNIT = "frames/s"
POLICY_SEED = 2
MAP_SEED = 1

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch
# from one ncu capture, valid only for the kernel source with this hash: the
# step kernel on the default workload's own 65,536 games (a one-pass capture
# of one launch); the sampler on 16,384 games, scaled by the games it
# processes (traffic grows in proportion).  Writes still dirty in the L2
# when a launch ends are not in its DRAM count.
NCU_TRAFFIC = {"kernel_sha1": "8302ad1d807f", "bytes_per_launch": 153810432.0 + 555577088.0,
               "warp_inst_per_launch": 118105197.0, "captured": "65,536 games (the bench's own launch)",
               "games": 65536}
SM_COUNT, SCHEDULERS_PER_SM = 152, 4  # one warp instruction per scheduler and clock
SAMPLE_NCU = {"kernel_sha1": "515d4f95a9c0", "bytes_per_launch": 4 * (133577216.0 + 3892480.0),
              "warp_inst_per_launch": 4 * 50199088.0, "captured": "16,384 games (x4)", "games": 65536}
# DRAM bytes of one frame of the ragged and mixed workloads, each in the form
# that the default batch rule picks (per-bucket launches for the four ragged
# buckets, summed; one work-list launch for the fifteen mixed buckets)
ROLLOUT_NCU = {"kernel_sha1": "8302ad1d807f",
               "1v1-131072-ragged15to30": {"form": "plain_buckets", "bytes_per_frame":
                                           (30479872.0 + 145809408.0 + 139023104.0 + 5467136.0)
                                           + (51041792.0 + 455997184.0 + 426810112.0 + 3328.0)},
               "mixed-32768-sides20to40": {"form": "plain_worklist", "bytes_per_frame": 128557824.0 + 867469568.0}}
FEATURE_NCU_TRAFFIC = {"kernel_sha1": "8af7d765f60a", "bytes_per_launch": 8 * (356319488.0 + 1554689024.0),
                       "captured": "8,192 games (x8)", "games": 65536}


def issue_roofline(launch_ms: float, G: int, clk, rec=None, source="gk_kernels.cu") -> dict | None:
    """An issue-bound kernel's second roofline: warp instructions per launch
    (ncu smsp__inst_executed.sum on the captured case, scaled by games) over
    the launch time, against SMs x schedulers x the SM clock sampled during
    the timed region."""
    rec = rec or NCU_TRAFFIC
    if rec["kernel_sha1"] != kernel_sha1(source) or G != rec["games"]:
        return None
    mhz = (clk.summary() or {}).get("sm_mhz")
    if not mhz:
        return None
    inst = rec["warp_inst_per_launch"]
    achieved = inst / (launch_ms * 1e-3)
    peak = SM_COUNT * SCHEDULERS_PER_SM * mhz * 1e6
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "warp instructions/s",
            "frac": achieved / peak, "warp_inst_per_launch": inst, "warp_inst_per_frame": inst / G,
            "source": f"ncu smsp__inst_executed.sum, {rec['captured']}; peak at the sampled {mhz} MHz"}


def kernel_sha1(name: str = "gk_kernels.cu") -> str:
    p = os.path.join(ROOT, "paper_2606_23348_gb300", "csrc", name)
    return hashlib.sha1(open(p, "rb").read()).hexdigest()[:12]


def algorithmic_bytes(env) -> int:
    """Bytes one step launch must move at minimum, from the library's layout:
    state read + write (int16 army, int8 owner, int8 terrain per cell),
    five per-player planes (int16 + 4 x int8) and the mask written, actions
    read and next actions written, reward / scoreboard / done written, game
    scalars read + written, game table read."""
    npad = env.npad.astype(np.int64)
    P = env.P.astype(np.int64)
    per_game = 2 * 4 * npad + 6 * P * npad + 4 * P + 4 * P + 4 * P + 8 * P + 1 + 2 * 32 + 32
    return int(per_game.sum())


def algorithmic_bytes_resident(env, K: int) -> float:
    """Per-frame bytes of a K-frame resident rollout: every frame's outputs,
    actions and scalars-free per-frame records, the state read and written
    once per K frames, and the actions log."""
    npad = env.npad.astype(np.int64)
    P = env.P.astype(np.int64)
    per_frame = 6 * P * npad + 4 * P + 4 * P + 8 * P + 1
    once = 2 * 4 * npad + 2 * 32 + 32 + 8 * P
    return float((per_frame + once / K).sum())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        busy = [x for x in sm if mx and x > 0.3 * mx] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def free_port() -> int:
    import socket
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def launch_ranks(n: int, argv=None) -> int:
    """Started with --gpus N > 1 outside a launcher: run this same command as
    N ranks on this node (one process per GPU, rendezvous on 127.0.0.1) and
    return their exit status.  Each rank steps its own games (global ids
    offset by rank); rank 0 prints the line, with n_gpus the ranks that
    reported."""
    argv = sys.argv[1:] if argv is None else argv
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.abspath(__file__), *argv]
    return subprocess.call(cmd)


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if _cuda() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)  # each rank's collectives on its own GPU
        dist.init_process_group(backend)
    return rank, world, local


def _cuda():
    import torch
    return torch.cuda.is_available()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _cuda() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _cuda() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle
def oracle_throughput(budget_s: float = 12.0, games: int = 1024):
    """The oracle as it stands, single-threaded, on the first `games` games of
    the workload for as many frames as fit in the time budget."""
    from oracle import OracleEnv
    from paper_2606_23348_gb300.workloads import workload
    H, W, mode, P, gen, _ = workload(WORKLOAD, G=games)
    orc = OracleEnv(H, W, mode, P, seed=MAP_SEED, **gen)
    frames = 0
    t0 = time.perf_counter()
    while True:
        orc.step(orc.policy(POLICY_SEED))
        frames += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return games * frames / el, {"games": games, "frames": frames, "seconds": round(el, 2)}


def run_reference(args, rank, world):
    """The oracle, single-threaded on the host: one step = one frame of the
    first 256 games of the workload (the same maps, policy and rules)."""
    if rank != 0:
        return
    from oracle import OracleEnv
    from paper_2606_23348_gb300.workloads import workload
    games = 256
    H, W, mode, P, gen, _ = workload(WORKLOAD, G=games)
    orc = OracleEnv(H, W, mode, P, seed=MAP_SEED, **gen)
    for _ in range(args.warmup):
        orc.step(orc.policy(POLICY_SEED))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.step(orc.policy(POLICY_SEED))
    el = time.perf_counter() - t0
    value = games * args.steps / el
    sample = f"first {games} games of the workload, one frame per step, single thread"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int16",
        "data": "synthetic (seeded counter-hash maps and policy)",
        "config": {"workload": WORKLOAD, "sample": sample, "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU path
def run_e2e(env, acts, args, world):
    """The same step through gen_step_host: pinned host actions copied in,
    every output and the next actions copied back, inside the timed region."""
    import torch

    from paper_2606_23348_gb300.generals import Outputs
    h_out = Outputs(env.layout, pin_host=True)
    h_act = acts.cpu().pin_memory()
    h_next = torch.empty_like(h_act).pin_memory()
    Ke = max(3, min(args.steps, args.e2e_steps))
    for _ in range(2):
        env.step_host(h_act, h_out, POLICY_SEED, h_next)
        h_act.copy_(h_next)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(Ke):
        env.step_host(h_act, h_out, POLICY_SEED, h_next)
        h_act.copy_(h_next)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    value = sum_over_ranks(float(env.G * Ke), world) / e2e_s
    return {"value": value, "unit": UNIT, "h2d_bytes_per_step": h_act.numel() * 4,
            "d2h_bytes_per_step": h_out.nbytes() + h_next.numel() * 4, "steps": Ke,
            "path": "gen_step_host (pinned host buffers, fused policy)"}


def run_ours(args, rank, world, local):
    import torch

    from paper_2606_23348_gb300.generals import GeneralsEnv, copy_peak_gbps
    from paper_2606_23348_gb300.workloads import shard, workload

    torch.cuda.set_device(local)
    H, W, mode, P, gen, _ = workload(WORKLOAD, G=args.games or None)
    G = int(H.shape[0])
    env = GeneralsEnv(H, W, mode, P, seed=MAP_SEED, game_id_base=shard(G, rank), **gen)
    if args.warps:
        env.set_launch(args.warps)
    out = env.new_outputs()
    acts = env.new_actions()
    stream = torch.cuda.current_stream()
    env.policy(POLICY_SEED, acts)
    # pre-roll to mid-game (players own territory, auto-resets under way),
    # then the untimed warm-up steps
    for _ in range(args.preroll + args.warmup):
        env.step_policy(acts, out, POLICY_SEED, acts)
    torch.cuda.synchronize()

    K = args.steps
    t_all = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        t_all[0].record(stream)
        for k in range(K):  # back to back: an event between two launches would break their chaining
            env.step_policy(acts, out, POLICY_SEED, acts)
        t_all[1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
    elapsed_ms = t_all[0].elapsed_time(t_all[1])
    # the roofline's launch duration: the timed region's average per launch
    # (its launches run back to back, chained); beside it, the duration of
    # one launch bracketed by events of its own, measured right after
    launch_ms = elapsed_ms / K
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(min(K, 20))]
    for a, b in ev:
        a.record(stream)
        env.step_policy(acts, out, POLICY_SEED, acts)
        b.record(stream)
    torch.cuda.synchronize()
    isolated_launch_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    elapsed_ms = max_over_ranks(elapsed_ms, world)
    frames_total = sum_over_ranks(float(G * K), world)
    value = frames_total / (elapsed_ms * 1e-3)

    # the same workload as 64-frame resident rollouts (every frame's outputs
    # written to a 64-frame buffer; state read and written once per rollout)
    resident = None
    if not args.no_resident:
        Kr = 64
        outK = env.new_outputs(frames=Kr)
        env.rollout(Kr, POLICY_SEED, acts, outK, None, 0)
        torch.cuda.synchronize()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        rounds = max(1, min(8, K // Kr))
        r0.record(stream)
        for _ in range(rounds):
            env.rollout(Kr, POLICY_SEED, acts, outK, None, 0)
        r1.record(stream)
        torch.cuda.synchronize()
        ms = r0.elapsed_time(r1) / (rounds * Kr)
        rb = algorithmic_bytes_resident(env, Kr)
        resident = {"frames_per_s": G / (ms * 1e-3), "ms_per_frame": ms, "rollout_frames": Kr,
                    "own_bytes_per_frame": rb, "hbm_frac_own_bytes": rb / (ms * 1e-3) / 1e9 / peaks()[0]}
        del outK

    # the configuration's full episode length: 2,000 more per-frame launches
    # of the same environment, timed as one region
    full = None
    if not args.no_resident and world == 1:
        n_full = 2000
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(n_full):
            env.step_policy(acts, out, POLICY_SEED, acts)
        f1.record(stream)
        torch.cuda.synchronize()
        ms = f0.elapsed_time(f1) / n_full
        full = {"frames": n_full, "frames_per_s": G / (ms * 1e-3), "ms_per_frame": ms,
                "hbm_frac": algorithmic_bytes(env) / (ms * 1e-3) / 1e9 / peaks()[0]}

    # e2e: the same step through the host-buffer entry point, copies timed
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(env, acts, args, world)

    nbytes = algorithmic_bytes(env)
    peak, peak_kind = peaks()
    achieved = nbytes / (launch_ms * 1e-3) / 1e9
    traffic = (NCU_TRAFFIC["bytes_per_launch"]
               if NCU_TRAFFIC["kernel_sha1"] == kernel_sha1() and G == NCU_TRAFFIC["games"] else None)
    own_peak = copy_peak_gbps(1 << 30, 5) if (rank == 0 and not args.no_copy_peak) else None

    # every other workload, each with its own timing and roofline (one GPU)
    configs = None
    if world == 1 and not args.no_configs:
        del out
        torch.cuda.empty_cache()
        configs = {}
        jobs = (("ragged_131072", lambda: rollout_record(args, "1v1-131072-ragged15to30", 64, 1, rank)),
                ("mixed_32768", lambda: rollout_record(args, "mixed-32768-sides20to40", 64, 1, rank)),
                ("served_256", lambda: served_record(args, args.served_seconds_default)),
                ("features", lambda: features_record(args, 65536, 10, rank)),
                ("sampler", lambda: sampler_record(args, 65536, 10, rank)),
                ("selfplay_512x512", lambda: selfplay_record(args, rank)))
        for name, job in jobs:
            t0 = time.perf_counter()
            try:
                configs[name] = job()
            except Exception as exc:  # one workload failing must not hide the others
                configs[name] = {"error": f"{type(exc).__name__}: {exc}"}
            configs[name]["bench_seconds"] = round(time.perf_counter() - t0, 1)
            torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle as it stands on every host core: one process per core on
        # disjoint game-id ranges (spawned, so safe after CUDA is up)
        from oracle.pool import parallel_throughput
        v1, sample = oracle_throughput(budget_s=args.cpu_seconds / 2)
        vn, procs, gf = parallel_throughput(WORKLOAD, MAP_SEED, POLICY_SEED, args.cpu_seconds / 2)
        cpu = {"value": vn, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"{procs} processes x 512 games of the workload (disjoint game ids) for "
                         f"{args.cpu_seconds / 2:.0f} s: {gf} game-frames",
               "single_thread": {"value": v1, "cores": 1,
                                 "sample": f"first {sample['games']} games x {sample['frames']} frames "
                                           f"({sample['seconds']} s)"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": elapsed_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int16",
            "data": "synthetic (seeded counter-hash maps, random legal policy, auto-reset)",
            "config": {"workload": WORKLOAD, "games_per_gpu": G, "preroll_frames": args.preroll, "board": "24x24",
                       "mode": "1v1",
                       "cities": 12, "mountains": 0.2, "policy": "uniform legal, split p=0.2",
                       "parallelism": f"replicas x{world} (disjoint game ids)",
                       "l2": "inputs larger than L2 (state 151 MB + outputs 529 MB per step)",
                       "launch": f"{args.warps or 8} warps per CTA, two games per warp"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "own_copy_kernel_gbps": own_peak, "algorithmic_bytes_per_launch": nbytes,
                         "launch_ms": launch_ms, "launch_ms_source": "timed region / K (launches back to back)",
                         "isolated_launch_ms": isolated_launch_ms, "kernel": "k_generals (fused step + policy)"},
            "issue_roofline": issue_roofline(launch_ms, G, clk),
            "cpu_baseline": cpu,
            "e2e": e2e,
            "resident_rollout_form": resident,
            "full_length_2000_frames": full,
            "configs": configs,
            "gpu_launches": K,
            "clocks": clk.summary(),
            "kernel_sha1": kernel_sha1(),
        }
        print(json.dumps(line), flush=True)


def rollout_record(args, name: str, K: int = 64, rounds: int = 1, rank: int = 0, batches=(1, 2),
                   rollouts: bool = True) -> dict:
    """A ragged or mixed workload in every launch form, each with both batch
    forms (one launch per size bucket on forked streams, and one persistent
    work-list launch over every bucket): per-frame launches, the same K frames
    as a CUDA graph, and one resident K-frame launch; frames/s and the HBM
    fraction of each (plain-form bytes per frame; the resident form also
    against its own bytes, the state moving once per K frames)."""
    import torch

    from paper_2606_23348_gb300.generals import GeneralsEnv
    from paper_2606_23348_gb300.workloads import shard, workload

    H, W, mode, P, gen, _ = workload(name)
    G = int(H.shape[0])
    env = GeneralsEnv(H, W, mode, P, seed=MAP_SEED, game_id_base=shard(G, rank), **gen)
    tune = env.autotune(steps=3) if getattr(args, "autotune", False) else "off"
    stream = torch.cuda.current_stream()
    acts = env.new_actions()
    env.policy(POLICY_SEED, acts)
    peak, peak_kind = peaks()
    nbytes = algorithmic_bytes(env)
    rb = algorithmic_bytes_resident(env, K)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    forms = {}
    out1 = env.new_outputs()
    outK = env.new_outputs(frames=K)
    for bname, batch in (("buckets", env.BATCH_BUCKETS), ("worklist", env.BATCH_WORKLIST)):
        if batch not in batches:
            continue
        env.set_batch_form(batch)
        for _ in range(max(3, args.warmup)):
            env.step_policy(acts, out1, POLICY_SEED, acts)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(rounds * K):
            env.step_policy(acts, out1, POLICY_SEED, acts)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (rounds * K)
        forms[f"plain_{bname}"] = {"frames_per_s": G / (ms * 1e-3), "ms_per_frame": ms,
                                   "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / peak,
                                   "launches_per_frame": len_buckets(env) if batch == 1 else 1}
        for fname, form in ((("graph", 1), ("resident", 0)) if rollouts else ()):
            for _ in range(2):
                env.rollout(K, POLICY_SEED, acts, outK, None, form)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(rounds):
                env.rollout(K, POLICY_SEED, acts, outK, None, form)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / (rounds * K)
            rec = {"frames_per_s": G / (ms * 1e-3), "ms_per_frame": ms, "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / peak}
            if form == 0:
                rec["own_bytes_per_frame"] = rb
                rec["hbm_frac_own_bytes"] = rb / (ms * 1e-3) / 1e9 / peak
            forms[f"{fname}_{bname}"] = rec
    buckets = len_buckets(env)
    del out1, outK, env
    torch.cuda.empty_cache()
    best_plain = max((k for k in ("plain_buckets", "plain_worklist") if k in forms),
                     key=lambda k: forms[k]["frames_per_s"])
    p = forms[best_plain]
    cap = ROLLOUT_NCU.get(name) if ROLLOUT_NCU["kernel_sha1"] == kernel_sha1() else None
    traffic = cap["bytes_per_frame"] if cap and cap["form"] == best_plain and G == int(workload(name)[0].shape[0]) \
        else None
    return {"workload": name, "games": G, "rollout_frames": K, "size_buckets": buckets, "autotune": tune,
            "forms": forms,
            "roofline": {"bound": "hbm", "achieved": nbytes / (p["ms_per_frame"] * 1e-3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": p["hbm_frac"], "traffic": traffic,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "algorithmic_bytes_per_frame": nbytes, "form": best_plain,
                         "kernel": "k_worklist" if best_plain == "plain_worklist" else "k_generals per bucket"}}


def run_rollout_workload(args, rank, world, local):
    """Ragged / mixed workloads: per-frame launches vs K-frame rollouts (CUDA
    graph of K launches, and one resident launch), bucketed by board size."""
    import torch
    torch.cuda.set_device(local)
    K = args.rollout
    rounds = max(1, args.steps // K)
    rec = rollout_record(args, args.workload, K, rounds, rank, (args.batch,) if args.batch else (1, 2),
                         not args.plain_only)
    forms = rec["forms"]
    best = max(forms, key=lambda k: forms[k]["frames_per_s"])
    if rank == 0:
        line = {
            "metric": METRIC, "value": forms[best]["frames_per_s"] * world, "unit": UNIT, "n_gpus": world,
            "steps": rounds * K, "warmup": args.warmup, "ms_per_step": forms[best]["ms_per_frame"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int16",
            "data": "synthetic (seeded counter-hash maps, random legal policy, auto-reset)",
            "config": {"workload": args.workload, "games_per_gpu": rec["games"], "rollout_frames": K,
                       "best_form": best, "size_buckets": rec["size_buckets"], "autotune": rec["autotune"],
                       "l2": "inputs larger than L2"},
            "roofline": rec["roofline"], "forms": forms,
            "gpu_launches": rounds * K * (rec["size_buckets"] if best.endswith("buckets") else 1),
        }
        print(json.dumps(line), flush=True)


SERVED_PARAMS = dict(seed=MAP_SEED, n_cities=-1, city_per_mille=30, city_army_min=40, city_army_max=50,
                     min_general_dist=0)
SERVED_SIM = dict(clients=256, mean_interarrival_ms=2.0, min_games=64, max_games=1024, min_side=15, max_side=40,
                  frac_1v1=0.4, frac_2v2=0.3, min_steps=20, max_steps=200, seed=11, policy_seed=POLICY_SEED,
                  budget_bytes=80 << 30, host_outputs=0, copy_outputs=0, open_loop=1)


def _served_row(st: dict) -> dict:
    keep = ("frames_per_s", "requests", "lat_p50_ms", "lat_p99_ms", "lat_mean_ms", "service_p50_ms", "service_p99_ms",
            "offered_requests_per_s", "tick_games_mean", "sessions_admitted", "sessions_waited",
            "sessions_waited_budget", "peak_bytes_in_use", "budget", "seconds", "tick_gpu_ms_mean",
            "tick_host_ms_mean")
    return {k: st[k] for k in keep}


def served_record(args, seconds: float, sweep: bool = False, admission: bool = False) -> dict:
    """The served workload: 256 actor clients with open-loop Poisson arrivals
    (mean 2 ms per client), each holding 64..1024 mixed games (40% 1v1, 30%
    2v2, 30% FFA-8) with sides 15..40, opening and closing sessions
    continuously, against an 80 GB admission budget; outputs stay on the
    device (GPU actors).  Beside it the plain bucketed step kernel on a batch
    of the same shape mix.  sweep: the same clients at 2, 4 and 8 times the
    offered load.  admission: an 80 GB run whose 96 clients' sessions (FFA-8,
    16,384 to 32,768 games each) outgrow the budget, so that admission
    defers."""
    import torch

    from paper_2606_23348_gb300.generals import GeneralsEnv
    from paper_2606_23348_gb300.server import simulate
    from paper_2606_23348_gb300.workloads import MOUNTAIN_THRESH_20PCT, shapes

    params = dict(SERVED_PARAMS, mountain_thresh=MOUNTAIN_THRESH_20PCT)
    rec = {"workload": "served-256-clients", "arrivals": "open loop, Poisson, mean 2 ms per client",
           "latency": "scheduled arrival to result in the client's buffers (queueing included); "
                      "service_* from submission",
           "nominal": _served_row(simulate(params, seconds=seconds, **SERVED_SIM))}
    if sweep:
        rec["load_sweep"] = []
        for mean in (8.0, 4.0, 1.0):  # a quarter, half and twice the nominal offered load
            st = simulate(params, seconds=seconds, **{**SERVED_SIM, "mean_interarrival_ms": mean})
            rec["load_sweep"].append({"mean_interarrival_ms": mean, **_served_row(st)})
    if admission:
        st = simulate(params, seconds=seconds, **{**SERVED_SIM, "clients": 96, "min_games": 16384,
                                                  "max_games": 32768, "frac_1v1": 0.0, "frac_2v2": 0.0,
                                                  "min_steps": 10, "max_steps": 40, "open_loop": 0})
        rec["admission_80gb"] = {"sessions": "96 clients x 16,384..32,768 FFA-8 games, sides 15..40, closed loop",
                                 **_served_row(st)}
    # the plain fixed-size kernel on a batch with the same shape distribution
    G = 256 * 544
    H, W, mode, P = shapes(G, (15, 40), ((0, 0.4), (1, 0.3), (2, 0.3)), seed=11)
    env = GeneralsEnv(H, W, mode, P, **params)
    out, acts = env.new_outputs(), env.new_actions()
    env.policy(POLICY_SEED, acts)
    for _ in range(max(3, args.warmup)):
        env.step_policy(acts, out, POLICY_SEED, acts)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    n = 20
    e0.record(stream)
    for _ in range(n):
        env.step_policy(acts, out, POLICY_SEED, acts)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    rec["plain_bucketed_kernel_same_mix"] = {"frames_per_s": G / (ms * 1e-3), "ms_per_frame": ms, "games": G}
    del env, out, acts
    torch.cuda.empty_cache()
    return rec


def run_served(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    rec = served_record(args, args.served_seconds, sweep=True, admission=True)
    nom = rec["nominal"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": nom["frames_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": int(nom["requests"]), "warmup": args.warmup, "ms_per_step": nom["lat_mean_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int16",
            "data": "synthetic (simulated actor clients, seeded maps, random legal policy)",
            "config": {"workload": "served-256-clients", **{k: v for k, v in SERVED_SIM.items() if k != "budget_bytes"},
                       "budget_gb": 80, "seconds": args.served_seconds},
            "served": rec, "latency_ms": {"p50": nom["lat_p50_ms"], "p99": nom["lat_p99_ms"]},
        }
        print(json.dumps(line), flush=True)


def feature_bytes_per_player_cell(hist: int, players: int) -> float:
    """Algorithmic HBM bytes of the feature builder per player and board cell:
    the float32 rows written, the memory read and written back (masks 1 B,
    last enemy army 2 B, its turn 4 B, one new own/enemy plane pair 4 B), the
    hist older plane pairs read (4 B each), and the board (4 B per cell)
    shared by the game's players."""
    C = 24 + 2 * hist
    return 4 * C + 7 + 4 * hist + 11 + 4.0 / players


def features_record(args, G: int, K: int, rank: int = 0, clk=None) -> dict:
    """Per frame: the fused step + policy, then the 38-channel feature tensor
    of every player (App. A) with its persistent memory and the 512-frame
    temporal tokens; the feature launch timed on its own."""
    import torch

    from paper_2606_23348_gb300.generals import GeneralsEnv
    from paper_2606_23348_gb300.workloads import shard, workload

    H, W, mode, P, gen, _ = workload("1v1-65536x24x24", G=G)
    hist, window = 7, 512
    env = GeneralsEnv(H, W, mode, P, seed=MAP_SEED, game_id_base=shard(G, rank), **gen)
    fb = env.features(hist, window)
    out, acts = env.new_outputs(), env.new_actions()
    fout, ser = fb.new_output(), fb.new_series()
    stream = torch.cuda.current_stream()
    env.policy(POLICY_SEED, acts)
    for _ in range(max(3, args.warmup)):
        env.step_policy(acts, out, POLICY_SEED, acts)
        fb.build(fout, ser)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    t_all = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    t_all[0].record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        env.step_policy(acts, out, POLICY_SEED, acts)
        ev[k][1].record(stream)
        fb.build(fout, ser)
        ev[k][2].record(stream)
    t_all[1].record(stream)
    torch.cuda.synchronize()
    elapsed_ms = t_all[0].elapsed_time(t_all[1])
    step_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    feat_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    cells = 2 * 576 * G
    # + temporal tokens per player: T - 1 ring entries read, one written, T written out (8 B each)
    nbytes = feature_bytes_per_player_cell(hist, 2) * cells + 2 * G * 8 * (2 * window)
    peak, peak_kind = peaks()
    achieved = nbytes / (feat_ms * 1e-3) / 1e9
    del fb, env, out, fout, ser
    torch.cuda.empty_cache()
    return {"workload": "features-65536x24x24" if G == 65536 else f"features-{G}x24x24", "games": G,
            "hist": hist, "channels": 24 + 2 * hist, "temporal_window": window,
            "frames_per_s": G * K / (elapsed_ms * 1e-3), "ms_per_frame": elapsed_ms / K,
            "step_launch_ms": step_ms, "feature_launch_ms": feat_ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": (FEATURE_NCU_TRAFFIC["bytes_per_launch"]
                                     if FEATURE_NCU_TRAFFIC["kernel_sha1"] == kernel_sha1("gk_features.cu")
                                     and G == FEATURE_NCU_TRAFFIC["games"] else None),
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "algorithmic_bytes_per_launch": nbytes, "launch_ms": feat_ms,
                         "kernel_sha1": kernel_sha1("gk_features.cu"),
                         "kernel": "k_features (38-channel feature tensor)"}}


def run_features(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    with ClockSampler(local) as clk:
        rec = features_record(args, args.games or 65536, args.steps, rank)
    if rank == 0:
        line = {
            "metric": "game frames/s with the 38-channel feature tensor and temporal tokens",
            "value": rec["frames_per_s"] * world, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": rec["ms_per_frame"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded counter-hash maps, random legal policy, auto-reset)",
            "config": {"workload": rec["workload"], "games_per_gpu": rec["games"], "hist": rec["hist"],
                       "channels": rec["channels"], "temporal_window": rec["temporal_window"],
                       "l2": "inputs larger than L2 (features 11.5 GB + memory 2.9 GB per frame)"},
            "roofline": rec["roofline"], "step_launch_ms": rec["step_launch_ms"], "gpu_launches": 2 * args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


SAMPLE_PREROLL = 256  # frames of the benchmark policy before the sampler is timed


def owned_player_cells(env) -> float:
    """Sum over games and players of the cells the player owns."""
    st = env.read_state()
    owner = st[1]
    return float(np.count_nonzero(owner >= 0))


def sampler_record(args, G: int, K: int, rank: int = 0, clk=None) -> dict:
    """Device self-play shape at mid-game: per frame, actions sampled from
    H x W x 9 logits (the sampler kernel), then the step (without the fused
    policy); the sampler launch timed on its own."""
    import torch

    from paper_2606_23348_gb300.generals import GeneralsEnv
    from paper_2606_23348_gb300.workloads import shard, workload

    H, W, mode, P, gen, _ = workload("1v1-65536x24x24", G=G)
    env = GeneralsEnv(H, W, mode, P, seed=MAP_SEED, game_id_base=shard(G, rank), **gen)
    out, acts = env.new_outputs(), env.new_actions()
    g = torch.Generator(device="cuda").manual_seed(1234 + rank)
    logits = torch.randn(int(env.layout.plane_cells) * 9, generator=g, device="cuda") * 2.0
    stream = torch.cuda.current_stream()
    env.policy(POLICY_SEED, acts)
    for _ in range(SAMPLE_PREROLL):  # to mid-game, so that players own territory
        env.step_policy(acts, out, POLICY_SEED, acts)
    for _ in range(max(3, args.warmup)):
        env.sample_actions(logits, POLICY_SEED, acts)
        env.step(acts, out)
    torch.cuda.synchronize()
    owned0 = owned_player_cells(env)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    t_all = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    t_all[0].record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        env.sample_actions(logits, POLICY_SEED, acts)
        ev[k][1].record(stream)
        env.step(acts, out)
        ev[k][2].record(stream)
    t_all[1].record(stream)
    torch.cuda.synchronize()
    elapsed_ms = t_all[0].elapsed_time(t_all[1])
    samp_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    step_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    # the logits a sampler must read (36 B per cell each player owns: legal entries lie only
    # there), board 4 B per cell once per game, actions 4 B per player; owned cells averaged
    # over the start and the end of the timed region
    owned = 0.5 * (owned0 + owned_player_cells(env))
    nbytes = 36.0 * owned + 4.0 * 576 * G + 4.0 * 2 * G
    # the same at DRAM-sector granularity: a cell's 36 logit bytes start at a
    # multiple of 4 bytes and always span two 32-byte sectors
    sector_bytes = 64.0 * owned + 4.0 * 576 * G + 4.0 * 2 * G
    peak, peak_kind = peaks()
    achieved = nbytes / (samp_ms * 1e-3) / 1e9
    del env, out, logits
    torch.cuda.empty_cache()
    return {"workload": "sample-65536x24x24" if G == 65536 else f"sample-{G}x24x24", "games": G,
            "preroll_frames": SAMPLE_PREROLL, "owned_cells_per_player": owned / (2 * G),
            "frames_per_s": G * K / (elapsed_ms * 1e-3), "ms_per_frame": elapsed_ms / K,
            "sampler_launch_ms": samp_ms, "step_launch_ms": step_ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": (SAMPLE_NCU["bytes_per_launch"]
                                     if SAMPLE_NCU["kernel_sha1"] == kernel_sha1("gk_sample.cu")
                                     and G == SAMPLE_NCU["games"] else None),
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "algorithmic_bytes_per_launch": nbytes, "launch_ms": samp_ms,
                         "sector_bytes_per_launch": sector_bytes,
                         "frac_of_sector_bytes": sector_bytes / (samp_ms * 1e-3) / 1e9 / peak,
                         "kernel": "k_sample_cta (H x W x 9 policy sampling, a CTA per game)"},
            "issue_roofline": None}  # needs the clocks of the timed region: the caller adds it


def run_sampling(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    with ClockSampler(local) as clk:
        rec = sampler_record(args, args.games or 65536, args.steps, rank, clk)
    rec["issue_roofline"] = issue_roofline(rec["sampler_launch_ms"], rec["games"], clk, SAMPLE_NCU, "gk_sample.cu")
    if rank == 0:
        line = {
            "metric": "game frames/s, actions sampled on the device from H x W x 9 logits",
            "value": rec["frames_per_s"] * world, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": rec["ms_per_frame"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 logits, int16 state",
            "data": "synthetic (seeded counter-hash maps, N(0, 2) logits, auto-reset)",
            "config": {"workload": rec["workload"], "games_per_gpu": rec["games"], "preroll_frames": SAMPLE_PREROLL,
                       "owned_cells_per_player": rec["owned_cells_per_player"],
                       "l2": "inputs larger than L2 (logits 2.7 GB)"},
            "roofline": rec["roofline"], "issue_roofline": rec["issue_roofline"],
            "step_launch_ms": rec["step_launch_ms"], "gpu_launches": 2 * args.steps, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def selfplay_record(args, rank: int = 0, T: int = 512, G: int = 512) -> dict:
    """The paper's rollout shape (512 environments x 512 steps) as a device
    self-play loop: per frame, actions sampled from H x W x 9 logits, the
    step, and the feature tensor with temporal tokens, with no host round
    trip; plain launches and the same T frames replayed as one CUDA graph."""
    import torch

    from paper_2606_23348_gb300.generals import GeneralsEnv
    from paper_2606_23348_gb300.workloads import shard, workload

    H, W, mode, P, gen, _ = workload("1v1-65536x24x24", G=G)
    env = GeneralsEnv(H, W, mode, P, seed=MAP_SEED, game_id_base=shard(G, rank), **gen)
    fb = env.features(7, 512)
    out, acts = env.new_outputs(), env.new_actions()
    x, tok = fb.new_output(), fb.new_series()
    g = torch.Generator(device="cuda").manual_seed(99 + rank)
    logits = torch.randn(int(env.layout.plane_cells) * 9, generator=g, device="cuda")
    stream = torch.cuda.Stream()

    def frame():
        env.sample_actions(logits, POLICY_SEED, acts)
        env.step(acts, out)
        fb.build(x, tok)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            frame()
    torch.cuda.synchronize()
    res = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(T):
            frame()
        e1.record(stream)
    torch.cuda.synchronize()
    res["plain"] = e0.elapsed_time(e1)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        for _ in range(T):
            frame()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        graph.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    res["graph"] = e0.elapsed_time(e1)

    def per_frame_ms(fn):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
            e0.record(stream)
            for _ in range(T):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / T

    # where a plain frame's time goes: the sampler and the step alone (after
    # the timed runs), the feature build as the rest
    parts = {"sample": per_frame_ms(lambda: env.sample_actions(logits, POLICY_SEED, acts)),
             "step": per_frame_ms(lambda: env.step(acts, out))}
    parts["features (rest of a plain frame)"] = res["plain"] / T - parts["sample"] - parts["step"]
    best = min(res, key=res.get)
    del graph, fb, env
    torch.cuda.empty_cache()
    return {"workload": "selfplay-512x512", "games": G, "frames": T, "hist": 7, "temporal_window": 512,
            "frames_per_s": G * T / (res[best] * 1e-3), "ms_per_frame": res[best] / T, "best_form": best,
            "forms": {k: {"ms_per_frame": v / T, "frames_per_s": G * T / (v * 1e-3)} for k, v in res.items()},
            "ms_per_frame_by_kernel": parts}


def run_selfplay(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    with ClockSampler(local) as clk:
        rec = selfplay_record(args, rank)
    if rank == 0:
        print(json.dumps({
            "metric": "game frames/s of a device self-play rollout (sample, step, features)",
            "value": rec["frames_per_s"] * world, "unit": "frames/s", "n_gpus": world, "steps": rec["frames"],
            "warmup": max(3, args.warmup), "ms_per_step": rec["ms_per_frame"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 logits and features, int16 state",
            "data": "synthetic (seeded counter-hash maps, N(0, 1) logits, auto-reset)",
            "config": {"workload": "selfplay-512x512", "games_per_gpu": rec["games"], "frames": rec["frames"],
                       "hist": 7, "temporal_window": 512, "l2": "fits in L2 (small batch; latency-bound)"},
            "forms": rec["forms"], "ms_per_frame_by_kernel": rec["ms_per_frame_by_kernel"],
            "gpu_launches": 3 * rec["frames"], "clocks": clk.summary()}), flush=True)


def run_batch_sweep(args, rank, world, local):
    """Frames/s of the default game shape (1v1, 24x24) at the environment
    counts of the paper's throughput table (Sec. V: 1,024 to 32,768 parallel
    environments) and at 65,536: one step + policy launch per frame, the same
    frames as a CUDA graph, and one resident multi-frame launch."""
    import torch

    from paper_2606_23348_gb300.generals import GeneralsEnv
    from paper_2606_23348_gb300.workloads import shard, workload

    torch.cuda.set_device(local)
    K = args.rollout
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    with ClockSampler(local) as clk:
        for G in (1024, 2048, 4096, 8192, 16384, 32768, 65536):
            H, W, mode, P, gen, _ = workload(WORKLOAD, G=G)
            env = GeneralsEnv(H, W, mode, P, seed=MAP_SEED, game_id_base=shard(G, rank), **gen)
            acts, out1 = env.new_actions(), env.new_outputs()
            env.policy(POLICY_SEED, acts)
            for _ in range(args.warmup):
                env.step_policy(acts, out1, POLICY_SEED, acts)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(K):
                env.step_policy(acts, out1, POLICY_SEED, acts)
            e1.record(stream)
            torch.cuda.synchronize()
            row = {"envs": G, "plain": G * K / (e0.elapsed_time(e1) * 1e-3)}
            del out1
            outK = env.new_outputs(frames=K)
            for name, form in (("graph", 1), ("resident", 0)):
                for _ in range(2):
                    env.rollout(K, POLICY_SEED, acts, outK, None, form)
                torch.cuda.synchronize()
                e0.record(stream)
                env.rollout(K, POLICY_SEED, acts, outK, None, form)
                e1.record(stream)
                torch.cuda.synchronize()
                row[name] = G * K / (e0.elapsed_time(e1) * 1e-3)
            rows.append({k: (v if k == "envs" else sum_over_ranks(v, world)) for k, v in row.items()})
            del env, outK
    best = max(rows, key=lambda r: max(r["plain"], r["graph"], r["resident"]))
    if rank == 0:
        print(json.dumps({
            "metric": "frames/s by environment count (step + policy, 1v1 24x24)",
            "value": max(best["plain"], best["graph"], best["resident"]), "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int16",
            "data": "synthetic (seeded counter-hash maps, random legal policy, auto-reset)",
            "config": {"workload": "sweep-1024to65536x24x24", "frames_per_form": K,
                       "l2": "small batches fit in L2 (latency-bound); the largest exceed it"},
            "rows": rows, "gpu_launches": None, "clocks": clk.summary()}), flush=True)


def _graph_us(fn, T: int, stream) -> float:
    """Device time per call of `fn`, T calls captured as one CUDA graph and
    replayed (best of three), so that host launch cost does not enter."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(3):
            fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for _ in range(T):
            fn()
    torch.cuda.synchronize()
    best = float("inf")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        with torch.cuda.stream(stream):
            e0.record(stream)
            g.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e3 / T)
    del g
    return best


def run_forms_sweep(args, rank, world, local):
    """Per-launch device time of every sampler form (warp per game, CTA per
    game, CTA per player) and both feature-builder forms (warp per game, CTA
    per player) on the default game shape (1v1 24x24) from 512 to 65,536
    games, at mid-game (256 frames of the benchmark policy), each form
    replayed as a CUDA graph of launches; and, at the self-play batch (512
    games), the sampler, step and feature launches alone and as a frame.
    Feature builds are timed as (step + build) - step, every build the first
    of its frame (the memory fold, the history ring full)."""
    import torch

    from paper_2606_23348_gb300.generals import GeneralsEnv
    from paper_2606_23348_gb300.workloads import shard, workload

    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    rows = []
    frame = {}
    with ClockSampler(local) as clk:
        for G in (512, 1024, 2048, 4096, 8192, 16384, 65536):
            T = 64 if G <= 8192 else 16
            H, W, mode, P, gen, _ = workload(WORKLOAD, G=G)
            env = GeneralsEnv(H, W, mode, P, seed=MAP_SEED, game_id_base=shard(G, rank), **gen)
            fb = env.features(7, 512)
            out, acts = env.new_outputs(), env.new_actions()
            x, tok = fb.new_output(), fb.new_series()
            env.policy(POLICY_SEED, acts)
            for f in range(STEP_PREROLL):
                env.step_policy(acts, out, POLICY_SEED, acts)
                if f >= STEP_PREROLL - 16:  # the feature history ring full
                    fb.build(x, tok)
            gen_ = torch.Generator(device="cuda").manual_seed(99 + rank)
            logits = torch.randn(int(env.layout.plane_cells) * 9, generator=gen_, device="cuda") * 2.0
            sampled = env.new_actions()
            fb.build(x, tok)
            torch.cuda.synchronize()
            row = {"games": G, "sampler_us": {}, "features_us": {}}
            for form, name in ((1, "warp_per_game"), (2, "cta_per_game"), (3, "cta_per_player")):
                env.set_sample_form(form)
                row["sampler_us"][name] = _graph_us(lambda: env.sample_actions(logits, POLICY_SEED, sampled), T,
                                                    stream)
            # a build folds the frame into the players' memory once per frame:
            # timed as (step + build) - step, so that every build is a frame's first
            step_us = _graph_us(lambda: env.step_policy(acts, out, POLICY_SEED, acts), T, stream)
            for form, name in ((1, "warp_per_game"), (2, "cta_per_player")):
                fb.set_form(form)
                row["features_us"][name] = _graph_us(lambda: (env.step_policy(acts, out, POLICY_SEED, acts),
                                                              fb.build(x, tok)), T, stream) - step_us
            env.set_sample_form(0)
            fb.set_form(0)
            if G == 512:
                frame = {"sample_us": _graph_us(lambda: env.sample_actions(logits, POLICY_SEED, sampled), T, stream),
                         "step_us": _graph_us(lambda: env.step(sampled, out), T, stream)}
                frame["features_us"] = _graph_us(lambda: (env.step(sampled, out), fb.build(x, tok)), T,
                                                 stream) - frame["step_us"]
                frame["frame_us"] = _graph_us(lambda: (env.sample_actions(logits, POLICY_SEED, sampled),
                                                       env.step(sampled, out), fb.build(x, tok)), T, stream)
            rows.append(row)
            del fb, env, out, x, tok, logits
            torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps({
            "metric": "us per launch by form and batch size (sampler, feature builder)", "value": None,
            "unit": "us", "n_gpus": world, "higher_is_better": False, "vs_baseline": None,
            "dtype": "f32 logits and features, int16 state",
            "data": "synthetic (seeded counter-hash maps, N(0, 2) logits, 256 policy frames)",
            "config": {"workload": "forms-512to65536x24x24", "hist": 7, "temporal_window": 512,
                       "timing": "CUDA graph of 64 launches (16 from 16,384 games), best of 3; features as "
                                 "(step + build) - step"},
            "rows": rows, "selfplay_512_frame_parts": frame, "gpu_launches": None,
            "clocks": clk.summary()}), flush=True)


def run_generator(args, rank, world, local):
    """Map generation throughput: gen_reset of every game of the default
    workload's shapes, for each generator option set."""
    import torch

    from paper_2606_23348_gb300.generals import GeneralsEnv
    from paper_2606_23348_gb300.workloads import workload

    torch.cuda.set_device(local)
    H, W, mode, P, gen, _ = workload(WORKLOAD)
    G = int(H.shape[0])
    res = {}
    for name, opts in (("manhattan", {}), ("bfs", dict(bfs_distance=1, min_general_dist=17)),
                       ("bfs+cap4", dict(bfs_distance=1, min_general_dist=1, max_general_dist=4)),
                       ("bfs+castle6", dict(bfs_distance=1, min_general_dist=17, castle_radius=6))):
        env = GeneralsEnv(H, W, mode, P, seed=MAP_SEED, **{**gen, **opts})
        out = env.new_outputs()
        stream = torch.cuda.current_stream()
        for _ in range(2):
            env.reset(out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        n = max(3, min(args.steps, 20))
        e0.record(stream)
        for _ in range(n):
            env.reset(out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        res[name] = {"maps_per_s": G / (ms * 1e-3), "ms_per_reset": ms}
        del env, out
    if rank == 0:
        print(json.dumps({"metric": "maps/s (reset of every game, outputs written)", "value": res["manhattan"]["maps_per_s"],
                          "unit": "maps/s", "n_gpus": world, "higher_is_better": True,
                          "config": {"workload": "generator-65536x24x24", "games": G}, "forms": res}), flush=True)


def len_buckets(env) -> int:
    """Size buckets of the batch (one launch each per frame)."""
    cls = set()
    for npad, p in zip(env.npad, env.P):
        edge = next(e for e in (256, 512, 768, 1024, 1536, 2048, 3072, 4096) if npad <= e)
        cls.add((edge, 2 if p <= 2 else 4 if p <= 4 else 8))
    return len(cls)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--warps", type=int, default=0, help="games per CTA (0 = library default)")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-copy-peak", action="store_true")
    ap.add_argument("--no-resident", action="store_true",
                    help="skip the resident-rollout and full-length (2,000 frames) figures")
    ap.add_argument("--workload", default=WORKLOAD, help="workload name (paper_2606_23348_gb300.workloads)")
    ap.add_argument("--games", type=int, default=0,
                    help="fewer games than the workload (profiling captures; 0 = the workload's count)")
    ap.add_argument("--rollout", type=int, default=64, help="frames per rollout (ragged / mixed workloads)")
    ap.add_argument("--autotune", action="store_true", help="autotune launch shapes first")
    ap.add_argument("--batch", type=int, default=0, choices=[0, 1, 2],
                    help="ragged / mixed workloads: 1 per-bucket launches only, 2 work-list launch only, 0 both")
    ap.add_argument("--plain-only", action="store_true",
                    help="ragged / mixed workloads: per-frame launches only (no graph or resident rollouts)")
    ap.add_argument("--served-seconds", type=float, default=10.0, help="measured window of the served workload")
    ap.add_argument("--served-seconds-default", type=float, default=3.0,
                    help="measured window of the served record inside the default line")
    ap.add_argument("--preroll", type=int, default=STEP_PREROLL,
                    help="benchmark-policy frames before the default workload's warm-up (mid-game state)")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload only (no ragged / mixed / served / features / sampler / self-play records)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(launch_ranks(args.gpus))
    rank, world, local = dist_setup(args.gpus)
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but {world} ranks were started")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        from paper_2606_23348_gb300.build import build_library
        if rank == 0:
            build_library()
        barrier(world)
        if args.workload == WORKLOAD:
            run_ours(args, rank, world, local)
        elif args.workload == "served-256-clients":
            run_served(args, rank, world, local)
        elif args.workload == "generator-65536x24x24":
            run_generator(args, rank, world, local)
        elif args.workload == "features-65536x24x24":
            run_features(args, rank, world, local)
        elif args.workload == "sample-65536x24x24":
            run_sampling(args, rank, world, local)
        elif args.workload == "selfplay-512x512":
            run_selfplay(args, rank, world, local)
        elif args.workload == "sweep-1024to65536x24x24":
            run_batch_sweep(args, rank, world, local)
        elif args.workload == "forms-512to65536x24x24":
            run_forms_sweep(args, rank, world, local)
        else:
            run_rollout_workload(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
