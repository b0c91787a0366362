"""Pins of the oracle's Philox4x32-10 and of the draw mapping of Algorithm 1 (CPU only)."""
import os

import numpy as np

from oracle import philox


def _kat(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_known_answer_vectors(golden_dir):
    rows = _kat(golden_dir)
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert list(philox.philox4x32_10(ctr, key)) == out


def test_vectorised_matches_scalar(golden_dir):
    for ctr, key, out in _kat(golden_dir):
        got = philox.philox4x32_10_many(np.array([ctr[0]]), ctr[1], ctr[2], ctr[3], key)[0]
        assert [int(v) for v in got] == out
    rng = np.random.default_rng(1)
    c = rng.integers(0, 2**32, size=(50, 4))
    k = rng.integers(0, 2**32, size=2)
    many = philox.philox4x32_10_many(c[:, 0], c[:, 1], c[:, 2], c[:, 3], k)
    # counters other than word 0 vary too: compare row by row with the scalar form
    for r in range(50):
        m1 = philox.philox4x32_10_many(np.array([c[r, 0]]), c[r, 1], c[r, 2], c[r, 3], k)[0]
        assert [int(v) for v in m1] == list(philox.philox4x32_10(c[r], k))
    assert many.shape == (50, 4)


def test_schedule_ranges_and_rates():
    N, p = 20, 0.1
    i, theta, coin = philox.schedule(20260209, 200000, N, p)
    assert i.min() == 0 and i.max() == N - 1
    counts = np.bincount(i, minlength=N) / len(i)
    assert np.all(np.abs(counts - 1.0 / N) < 0.005)
    assert abs(theta.mean() - p) < 0.003
    assert abs(coin.mean() - 1.0 / N) < 0.003


def test_schedule_p_one_is_always_prox():
    _, theta, _ = philox.schedule(7, 1000, 10, 1.0)
    assert theta.all()


def test_subset_index_is_high_word_product():
    w = philox.words(99, 0, 64)
    i, _, _ = philox.schedule(99, 64, 7, 0.5)
    for k in range(64):
        assert i[k] == (int(w[k, 0]) * 7) >> 32


def test_threshold_exact():
    assert philox.skip_threshold(0.5) == 2**31
    assert philox.skip_threshold(0.25) == 2**30
    assert philox.skip_threshold(1.0) == 2**32


def test_uniform01_open_interval():
    u = philox.uniform01(3, 1001)
    assert u.shape == (1001,)
    assert u.min() > 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.03
