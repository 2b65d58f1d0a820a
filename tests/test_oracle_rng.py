"""Pins of the oracle's counter-based generators and initialisation (CPU only)."""
import math
import os

import numpy as np

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def test_splitmix64_known_outputs():
    for seed, i, out in _rows("splitmix64_kat.txt"):
        assert rng.splitmix64(int(seed), int(i)) == int(out)


def test_philox_known_answer_vectors():
    for r in _rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in r]
        out = rng.philox4x32_10(np.array([v[0:4]], dtype=np.uint64), np.array([v[4:6]], dtype=np.uint64))[0]
        assert [int(x) for x in out] == v[6:10]


def test_sample_indices_range_and_uniformity():
    n = 1000
    idx = rng.sample_indices(seed=42, net=1, step=7, batch=200000, population=n)
    assert idx.min() >= 0 and idx.max() < n
    counts = np.bincount(idx, minlength=n)
    chi2 = float(((counts - 200.0) ** 2 / 200.0).sum())
    assert chi2 < n + 6 * math.sqrt(2 * n)          # ~6 sigma of a chi^2(n-1)
    # different steps / nets give different streams
    a = rng.sample_indices(42, 1, 7, 64, 1 << 31)
    b = rng.sample_indices(42, 1, 8, 64, 1 << 31)
    c = rng.sample_indices(42, 2, 7, 64, 1 << 31)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


def test_sample_index_is_word_of_philox_block():
    # sample s uses word s%4 of the block with counter (s//4, step, net, 0)
    seed = 0x123456789ABCDEF
    idx = rng.sample_indices(seed, 2, 5, 9, 1 << 31)
    ctr = np.array([[2, 5, 2, 0]], dtype=np.uint64)
    key = np.array([[seed & 0xFFFFFFFF, seed >> 32]], dtype=np.uint64)
    w = rng.philox4x32_10(ctr, key)[0]
    assert idx[8] == int(w[0]) >> 1          # population 2^31: index = u32 >> 1


def test_xavier_bounds_and_moments():
    net = rng.xavier_net(seed=3, net=2, n_in=64, width=64, layers=4)
    a0 = math.sqrt(6.0 / 128)
    W0 = net["W"][0]
    assert W0.shape == (64, 64) and np.all(np.abs(W0) <= a0)
    assert np.array_equal(W0, W0.astype(np.float32).astype(np.float64))
    allw = np.concatenate([w.reshape(-1) for w in net["W"][1:]])
    assert abs(allw.mean()) < 0.02 and abs(allw.var() / (a0 * a0 / 3.0) - 1.0) < 0.05
    assert all(np.all(b == 0) for b in net["b"]) and net["bh"] == 0.0
    assert np.all(np.abs(net["wh"]) <= math.sqrt(6.0 / 65))


def test_ffm_increments_are_gaussian_with_sigma():
    sigma, E = 3.0, 1024
    q = rng.ffm_increments(seed=9, level=0, m=4000, sigma=sigma, extent=E)
    s = q.astype(np.int64)
    s = np.where(s >= 1 << 31, s - (1 << 32), s).astype(np.float64)
    B = s * E / 2.0 ** 32
    assert abs(B.mean()) < 0.1
    assert abs(B.std() / sigma - 1.0) < 0.03
    # fraction within one sigma of a normal distribution
    assert abs(np.mean(np.abs(B) < sigma) - 0.6827) < 0.02
