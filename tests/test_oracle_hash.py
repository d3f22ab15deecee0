"""The counter-based hash pinned to SplitMix64's published outputs.

SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) seeded with 1234567 yields the
sequence below in the reference implementation distributed with the
xoshiro/xoroshiro generators; the oracle's n-th stream output must match.
"""
import numpy as np

from oracle import draw, key, sm

KAT_SEED = 1234567
KAT = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
       16408922859458223821]


def test_splitmix64_published_vectors():
    assert [sm(KAT_SEED, n) for n in range(5)] == KAT


def test_draw_is_high_half():
    assert draw(KAT_SEED, 0) == KAT[0] >> 32
    assert draw(KAT_SEED, 4) == KAT[4] >> 32


def test_key_nests_streams():
    # key(s, a, b, c) is the c-th output of the stream seeded by the b-th output
    # of the stream seeded by the a-th output of the stream seeded by s
    k1 = sm(KAT_SEED, 3)
    assert key(KAT_SEED, 3, 0, 0) == sm(sm(k1, 0), 0)
    assert key(KAT_SEED, 0, 1, 2) == sm(sm(KAT[0], 1), 2)


def test_draw_uniform_chi_square():
    k = key(99, 1, 2, 3)
    u = np.array([draw(k, i) for i in range(20000)], dtype=np.uint64)
    hist = np.bincount((u >> np.uint64(28)).astype(np.int64), minlength=16)
    exp = len(u) / 16
    chi2 = float(((hist - exp) ** 2 / exp).sum())
    assert chi2 < 37.7  # 99.9th percentile of chi-square with 15 dof
