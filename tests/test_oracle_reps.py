"""Pins for the representative sampler (Section 4, fixed-size reading).

* SplitMix64's published output stream for seed 1234567 (the known-answer
  values printed with the reference implementation by Vigna / Steele et al.).
* Distinct ids, sorted, inside [0, n).
* Uniformity: inclusion frequencies over many seeds agree with n_r / n
  (Section 4's selection probability) within a chi-square bound.
* The stored fixture ``tests/golden/reps_n16384_nr128_seed2.txt`` (written by
  ``tests/golden/make_golden.py`` from the oracle alone).
"""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_known_answer():
    g = oracle.SplitMix64(1234567)
    got = [g.next() for _ in range(5)]
    assert got == [
        6457827717110365317,
        3203168211198807973,
        9817491932198370423,
        4593380528125082431,
        16408922859458223821,
    ]


def test_below_is_in_range_and_rejects():
    g = oracle.SplitMix64(7)
    vals = [g.below(3) for _ in range(3000)]
    assert set(vals) == {0, 1, 2}
    counts = np.bincount(vals)
    assert np.all(np.abs(counts - 1000) < 150)
    # bound 1 always returns 0; bound 2^63+1 exercises the rejection limit
    assert all(g.below(1) == 0 for _ in range(10))
    big = (1 << 63) + 1
    assert all(0 <= g.below(big) < big for _ in range(100))


def test_sample_basic_properties():
    for n, n_r, seed in [(10, 10, 0), (1000, 31, 5), (1 << 20, 1024, 2), (7, 1, 3)]:
        r = oracle.sample_reps(n, n_r, seed)
        assert len(r) == n_r
        assert np.all(np.diff(r) > 0)
        assert r[0] >= 0 and r[-1] < n
    assert oracle.sample_reps(10, 10, 0).tolist() == list(range(10))


def test_sample_inclusion_uniform():
    n, n_r, trials = 40, 8, 4000
    hits = np.zeros(n)
    for s in range(trials):
        hits[oracle.sample_reps(n, n_r, 1000 + s)] += 1
    expected = trials * n_r / n
    chi2 = float(((hits - expected) ** 2 / expected).sum())
    # 39 degrees of freedom; P(chi2 > 80) < 1e-4 (the true variance is a
    # little smaller than the chi-square model assumes, so this is loose)
    assert chi2 < 80.0, chi2


def test_sample_seed_changes_sample():
    a = oracle.sample_reps(100000, 300, 1)
    b = oracle.sample_reps(100000, 300, 2)
    assert not np.array_equal(a, b)
    np.testing.assert_array_equal(a, oracle.sample_reps(100000, 300, 1))


def test_sample_golden_fixture():
    path = os.path.join(GOLDEN, "reps_n16384_nr128_seed2.txt")
    want = np.loadtxt(path, dtype=np.int64)
    np.testing.assert_array_equal(oracle.sample_reps(16384, 128, 2), want)
