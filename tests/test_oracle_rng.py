"""Pins of the oracle's SplitMix64 streams (published reference outputs, invariants)."""

import numpy as np

from oracle import rng


def test_splitmix64_reference_outputs():
    # The first three outputs of SplitMix64 seeded with 0, as published with the
    # generator's reference implementation (Steele, Lea & Flood 2014; Vigna's splitmix64.c).
    out = rng.splitmix_output(np.uint64(0), np.arange(3, dtype=np.uint64))
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_access_matches_sequential_state():
    # Output i computed directly equals stepping the state i+1 times.
    key = rng.stream_key(7, rng.TAG_PERM)
    direct = rng.splitmix_output(key, np.arange(100, dtype=np.uint64))
    state = int(key)
    seq = []
    for _ in range(100):
        state = (state + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
        seq.append(int(rng.mix64(np.array([state], np.uint64))[0]))
    assert [int(v) for v in direct] == seq


def test_uniform_range_and_moments():
    u = rng.unit_uniform(rng.draws(3, rng.TAG_XVAL, 200000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005
    assert abs(u.var() - 1.0 / 12.0) < 0.002
    hist, _ = np.histogram(u, bins=20, range=(0, 1))
    expected = len(u) / 20
    chi2 = ((hist - expected) ** 2 / expected).sum()
    assert chi2 < 60.0      # 19 dof; p ~ 1e-6


def test_streams_and_seeds_differ():
    a = rng.draws(0, rng.TAG_SIGMA, 1000)
    b = rng.draws(0, rng.TAG_PERM, 1000)
    c = rng.draws(1, rng.TAG_SIGMA, 1000)
    assert len(np.intersect1d(a, b)) == 0
    assert len(np.intersect1d(a, c)) == 0
