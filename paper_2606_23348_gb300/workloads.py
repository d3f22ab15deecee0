"""Seeded synthetic workloads (per-game board shapes and modes).

This module holds no game arithmetic: it only draws the per-game sizes and
modes of a workload with numpy's seeded generator, so that the CUDA path and
the CPU oracle are handed identical inputs.  Maps and actions themselves are
drawn inside each side from the counter-based hash.

Workloads follow the shapes of the paper's self-play games (Section IV-A:
H x W grids up to 23 x 23, 20% mountains, neutral castles with 40-50 units);
the paper names no public dataset.
"""
from __future__ import annotations

import numpy as np

MOUNTAIN_THRESH_20PCT = 858993459  # floor(0.2 * 2^32)

# name -> description; sizes are per game.  "auto" general distance is
# floor((H + W) / 3): 10 on 15 x 15, 16 on 24 x 24.
WORKLOADS = {
    "1v1-64x15x15": dict(G=64, side=(15, 15), modes=((0, 1.0),), n_cities=8, city_per_mille=0, frames=500),
    "1v1-65536x24x24": dict(G=65536, side=(24, 24), modes=((0, 1.0),), n_cities=12, city_per_mille=0,
                            frames=2000),
    "1v1-131072-ragged15to30": dict(G=131072, side=(15, 30), modes=((0, 1.0),), n_cities=-1, city_per_mille=20,
                                    frames=64),
    "mixed-32768-sides20to40": dict(G=32768, side=(20, 40), modes=((0, 0.4), (1, 0.3), (2, 0.3)), n_cities=-1,
                                    city_per_mille=30, frames=1000),
}


def shapes(G: int, side=(15, 15), modes=((0, 1.0),), seed: int = 0, ffa_players: int = 8):
    """Per-game (H, W, mode, n_players) int32 arrays.

    ``side`` = (lo, hi): H and W independently uniform in [lo, hi].
    ``modes`` = ((mode, fraction), ...): the first round(fraction * G) games of
    each mode, then shuffled with the same generator.
    """
    rng = np.random.default_rng(seed)
    lo, hi = side
    if lo == hi:
        H = np.full(G, lo, np.int32)
        W = np.full(G, lo, np.int32)
    else:
        H = rng.integers(lo, hi + 1, size=G).astype(np.int32)
        W = rng.integers(lo, hi + 1, size=G).astype(np.int32)
    mode = np.zeros(G, np.int32)
    start = 0
    for k, (m, frac) in enumerate(modes):
        n = G - start if k == len(modes) - 1 else int(round(frac * G))
        mode[start:start + n] = m
        start += n
    if len(modes) > 1:
        rng.shuffle(mode)
    n_players = np.where(mode == 0, 2, np.where(mode == 1, 4, ffa_players)).astype(np.int32)
    return H, W, mode, n_players


def workload(name: str, seed: int = 0, G: int | None = None):
    """Shapes and generator parameters of a named workload (optionally fewer games)."""
    w = WORKLOADS[name]
    n = w["G"] if G is None else G
    H, W, mode, n_players = shapes(n, w["side"], w["modes"], seed=seed)
    gen = dict(mountain_thresh=MOUNTAIN_THRESH_20PCT, n_cities=w["n_cities"], city_per_mille=w["city_per_mille"],
               city_army_min=40, city_army_max=50, min_general_dist=0)
    return H, W, mode, n_players, gen, w["frames"]


def random_actions(rng: np.random.Generator, N: np.ndarray, P: int = 8, p_pass: float = 0.1,
                   p_bad: float = 0.05) -> np.ndarray:
    """Arbitrary (mostly in-range) action indices [G][P] for fuzzing the validator."""
    G = N.shape[0]
    a = (rng.random((G, P)) * (9 * N[:, None])).astype(np.int64)
    a[rng.random((G, P)) < p_pass] = 0
    bad = rng.random((G, P)) < p_bad
    a[bad] = rng.integers(-5, 5, size=int(bad.sum())) + np.where(rng.random(int(bad.sum())) < 0.5, 0,
                                                                9 * np.repeat(N, P).reshape(G, P)[bad])
    return a.astype(np.int32)


def shard(games_per_rank: int, rank: int) -> int:
    """Global id of a rank's first game: ranks own disjoint, contiguous id
    ranges, so no exchange is needed while stepping (weak scaling)."""
    return int(rank) * int(games_per_rank)
