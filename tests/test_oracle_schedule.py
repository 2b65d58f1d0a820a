"""Pins of the oracle's training schedules (CPU only): subset resampling (Appendix E) and
the regressor populations of the sparsity ablation (Appendix C).

Resampling: every batch of an interval lies inside that interval's subset (enumerated
element by element), a subset holds at most interval x batch distinct candidates, and
consecutive intervals draw different subsets.  Populations: enumerated by brute force from
the input voxel set -- blocked samples are the voxels of the leaves, dense samples the
voxels of the domain's box in x-major order, and both take the voxel's value where it is
active and the background elsewhere.
"""
import numpy as np

from fixtures import workload
from oracle import codec, rng, vdb


def test_resampled_batches_come_from_their_interval_subset():
    seed, net, B, R, pop = 5, 2, 64, 10, 100_000
    key = np.array([[seed & 0xFFFFFFFF, seed >> 32]], dtype=np.uint64)
    for r in range(3):
        subset = set()
        for p in range(R * B):   # the interval's subset, element by element
            w = rng.philox4x32_10(np.array([[p // 4, r, net, 1]], dtype=np.uint64), key)[0, p % 4]
            subset.add(int((int(w) * pop) >> 32))
        seen = set()
        for t in range(r * R + 1, (r + 1) * R + 1):
            idx = rng.subset_indices(seed, net, t, B, R, pop)
            assert set(idx.tolist()) <= subset
            seen |= set(idx.tolist())
        assert len(seen) <= R * B
        if r == 0:
            first = subset
        else:
            assert len(subset & first) < 0.1 * len(subset)   # a fresh subset
    # without resampling, ten consecutive batches spread over far more of the population
    fresh = set()
    for t in range(1, R + 1):
        fresh |= set(rng.sample_indices(seed, net, t, B, pop).tolist())
    assert len(fresh) > 0.9 * R * B


def _grid(name):
    ijk, val, _ = workload(name)
    ijk, val = ijk.numpy().astype(np.int64), val.numpy()
    return vdb.build(ijk, val), {tuple(c): float(v) for c, v in zip(ijk.tolist(), val.tolist())}


def test_blocked_population_brute_force():
    for name, cls in (("sphere32", 0), ("fog64", 1)):
        g, truth = _grid(name)
        m = codec.init_model(g, cls, 3.0, codec.default_opts(width=[8, 8, 8], layers=[1, 1, 1]))
        idx = np.arange(0, g["leaf_origin"].shape[0] * 512, 7)
        ijk, tgt = codec.regressor_population(g, m, idx, codec.BLOCKED)
        for i, c, t in zip(idx.tolist(), ijk.tolist(), tgt.tolist()):
            o = g["leaf_origin"][i // 512].tolist()
            off = i % 512
            assert tuple(c) == (o[0] + off // 64, o[1] + (off // 8) % 8, o[2] + off % 8)
            v = truth.get(tuple(c))
            want = (v / 3.0 if cls == 0 else v) if v is not None else (1.0 if cls == 0 else 0.0)
            assert t == want


def test_dense_population_brute_force():
    g, truth = _grid("sphere32")
    m = codec.init_model(g, 0, 3.0, codec.default_opts(width=[8, 8, 8], layers=[1, 1, 1]))
    E = 1 << m["log2_extent"]
    idx = np.arange(E ** 3)
    ijk, tgt = codec.regressor_population(g, m, idx, codec.DENSE)
    o = m["origin"]
    assert np.array_equal(ijk[1], o + [0, 0, 1]) and np.array_equal(ijk[E], o + [0, 1, 0])
    assert np.array_equal(ijk[E * E], o + [1, 0, 0])
    active = np.array([tuple(c) in truth for c in ijk.tolist()])
    assert active.sum() == len(truth)                     # every input voxel, once
    assert np.all(tgt[~active] == 1.0)                    # background +w, scaled
    sel = np.nonzero(active)[0][::97]
    assert all(tgt[i] == truth[tuple(ijk[i].tolist())] / 3.0 for i in sel)
