"""Pins of the oracle's VDB tree build against brute-force enumeration (CPU only)."""
import numpy as np
import pytest

from oracle import vdb


def _random_voxels(seed, n, lo, hi):
    r = np.random.default_rng(seed)
    ijk = np.unique(r.integers(lo, hi, (n, 3)), axis=0)
    r.shuffle(ijk)
    return ijk, r.standard_normal(ijk.shape[0]).astype(np.float32)


@pytest.mark.parametrize("lo,hi", [(0, 64), (3990, 4210), (1 << 20, (1 << 20) + 300)])
def test_build_matches_brute_force(lo, hi):
    ijk, val = _random_voxels(1, 3000, lo, hi)
    g = vdb.build(ijk, val)
    # canonical order: the key tuple written out field by field
    def tkey(p):
        i, j, k = map(int, p)
        return (i >> 12, j >> 12, k >> 12, (i >> 7) & 31, (j >> 7) & 31, (k >> 7) & 31,
                (i >> 3) & 15, (j >> 3) & 15, (k >> 3) & 15, i & 7, j & 7, k & 7)
    order = sorted(range(len(ijk)), key=lambda a: tkey(ijk[a]))
    assert np.array_equal(g["ijk"], ijk[order])
    assert np.array_equal(g["val"], val[order])
    # nodes: every distinct aligned origin, once
    for name, mask in (("leaf_origin", ~7), ("l1_origin", ~127), ("l2_origin", ~4095)):
        want = {tuple(int(x) for x in (p & mask)) for p in ijk}
        got = [tuple(int(x) for x in p) for p in g[name]]
        assert len(got) == len(set(got)) == len(want) and set(got) == want
    # leaf masks: bit set exactly at the voxel offsets of that leaf
    leaf_index = {tuple(int(x) for x in p): n for n, p in enumerate(g["leaf_origin"])}
    expect = np.zeros_like(g["leaf_mask"])
    for p in ijk:
        n = leaf_index[tuple(int(x) for x in (p & ~7))]
        off = ((int(p[0]) & 7) << 6) | ((int(p[1]) & 7) << 3) | (int(p[2]) & 7)
        expect[n, off // 64] |= np.uint64(1) << np.uint64(off % 64)
    assert np.array_equal(expect, g["leaf_mask"])
    # level-1 child masks: one bit per child leaf at its slot
    l1_index = {tuple(int(x) for x in p): n for n, p in enumerate(g["l1_origin"])}
    expect = np.zeros_like(g["l1_mask"])
    for p in g["leaf_origin"]:
        n = l1_index[tuple(int(x) for x in (p & ~127))]
        s = ((int(p[0]) >> 3 & 15) << 8) | ((int(p[1]) >> 3 & 15) << 4) | (int(p[2]) >> 3 & 15)
        expect[n, s // 64] |= np.uint64(1) << np.uint64(s % 64)
    assert np.array_equal(expect, g["l1_mask"])
    # popcounts
    assert vdb.popcount(g["leaf_mask"]) == len(ijk)
    assert vdb.popcount(g["l1_mask"]) == g["leaf_origin"].shape[0]
    assert vdb.popcount(g["l2_mask"]) == g["l1_origin"].shape[0]
    # level-1 origins recovered from the level-2 child masks alone
    assert np.array_equal(vdb.l1_origins_from_upper(g["l2_origin"], g["l2_mask"]), g["l1_origin"])


def test_build_rejects_duplicates_and_range():
    ijk = np.array([[1, 2, 3], [4, 5, 6], [1, 2, 3]])
    with pytest.raises(vdb.DuplicateVoxel):
        vdb.build(ijk, np.zeros(3))
    with pytest.raises(ValueError):
        vdb.build(np.array([[-1, 0, 0]]), np.zeros(1))
    with pytest.raises(ValueError):
        vdb.build(np.array([[1 << 21, 0, 0]]), np.zeros(1))


def test_build_empty():
    g = vdb.build(np.zeros((0, 3), np.int64), np.zeros(0))
    assert g["n"] == 0 and g["leaf_origin"].shape[0] == 0 and g["l2_origin"].shape[0] == 0


def test_domain_is_power_of_two_cover():
    o, l = vdb.domain(np.array([[22, 22, 22], [106, 106, 106]]))
    assert list(o) == [0, 0, 0] and l == 7
    o, l = vdb.domain(np.array([[3990, 100, 5000], [4210, 120, 5001]]))
    assert list(o) == [3968, 0, 4992] and l == 8   # extent 4224 - 3968 = 256
