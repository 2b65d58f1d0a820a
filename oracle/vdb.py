"""VDB [Hash,5,4,3] tree from sparse voxels (Section 3.1).

Levels: leaf (level 0) = 8^3 voxels with an active mask a_0; level-1 internal
node = 16^3 children (128^3 voxels) with child mask c_1; level-2 internal node
= 32^3 children (4096^3 voxels) with child mask c_2; root = sparse map of
level-2 nodes.  By default every input voxel stays explicit and the active masks of
the internal nodes are empty.  With tile pruning (tolerance tol >= 0, Section 3.1:
tile values stand for constant regions), a leaf whose 512 voxels are all active and
whose values span at most tol (FP32 max - min <= tol) becomes an active tile of its
level-1 node: bit `slot` of the level-1 active mask a_1, tile value the FP32 midpoint
(min + max) * 0.5.  The explicit grid keeps such a tile expanded as its leaf (so the
leaf arrays, samplers and canonical order are unchanged) with every voxel carrying the
tile value.

Canonical order is that of the dense node layouts: lexicographic on
(level-2 key, level-1 slot, leaf slot, voxel offset) with
  level-2 key = (i>>12, j>>12, k>>12)
  level-1 slot = ((i>>7)&31)<<10 | ((j>>7)&31)<<5 | ((k>>7)&31)
  leaf slot    = ((i>>3)&15)<<8  | ((j>>3)&15)<<4 | ((k>>3)&15)
  voxel offset = (i&7)<<6 | (j&7)<<3 | (k&7).
Bit b of a mask is bit (b & 63) of 64-bit word (b >> 6).
Coordinates must lie in [0, 2^21).
"""
from __future__ import annotations

import numpy as np

COORD_LIMIT = 1 << 21


class DuplicateVoxel(ValueError):
    pass


def canonical_key(ijk: np.ndarray) -> np.ndarray:
    i, j, k = (ijk[:, d].astype(np.int64) for d in range(3))
    l2 = ((i >> 12) << 18) | ((j >> 12) << 9) | (k >> 12)
    l1 = (((i >> 7) & 31) << 10) | (((j >> 7) & 31) << 5) | ((k >> 7) & 31)
    lf = (((i >> 3) & 15) << 8) | (((j >> 3) & 15) << 4) | ((k >> 3) & 15)
    off = ((i & 7) << 6) | ((j & 7) << 3) | (k & 7)
    return (l2 << 36) | (l1 << 21) | (lf << 9) | off


def _set_bits(words: np.ndarray, row: np.ndarray, bit: np.ndarray):
    bit = np.asarray(bit, dtype=np.int64)
    np.bitwise_or.at(words, (np.asarray(row, dtype=np.int64), bit >> 6),
                     np.left_shift(np.uint64(1), (bit & 63).astype(np.uint64)))


def test_bit(words: np.ndarray, row, bit) -> np.ndarray:
    row = np.asarray(row, dtype=np.int64)
    bit = np.asarray(bit, dtype=np.int64)
    w = words[row, bit >> 6]
    return ((w >> (bit & 63).astype(np.uint64)) & np.uint64(1)).astype(bool)


def popcount(words: np.ndarray) -> int:
    return int(sum(bin(int(x)).count("1") for x in words.reshape(-1)))


def build(ijk, val, tile_tol: float | None = None) -> dict:
    """Sort voxels canonically and build the masks of every level (and, with a tolerance,
    the active tiles of level 1)."""
    ijk = np.asarray(ijk, dtype=np.int64).reshape(-1, 3)
    val = np.asarray(val, dtype=np.float32).reshape(-1)
    if ijk.shape[0] != val.shape[0]:
        raise ValueError("ijk and val sizes differ")
    if ijk.size and (ijk.min() < 0 or ijk.max() >= COORD_LIMIT):
        raise ValueError("coordinates must lie in [0, 2^21)")
    key = canonical_key(ijk)
    order = np.argsort(key, kind="stable")
    key, ijk, val = key[order], ijk[order], val[order]
    if key.size > 1 and np.any(key[1:] == key[:-1]):
        raise DuplicateVoxel("duplicate voxel")
    n = key.size
    leaf_key, leaf_first = np.unique(key >> 9, return_index=True)
    l1_key, l1_first = np.unique(key >> 21, return_index=True)
    l2_key, l2_first = np.unique(key >> 36, return_index=True)
    leaf_of_vox = np.searchsorted(leaf_key, key >> 9)
    l1_of_leaf = np.searchsorted(l1_key, leaf_key >> 12)
    l2_of_l1 = np.searchsorted(l2_key, l1_key >> 15)
    leaf_mask = np.zeros((leaf_key.size, 8), dtype=np.uint64)
    _set_bits(leaf_mask, leaf_of_vox, key & 511)
    l1_mask = np.zeros((l1_key.size, 64), dtype=np.uint64)
    _set_bits(l1_mask, l1_of_leaf, (leaf_key & 4095))
    l2_mask = np.zeros((l2_key.size, 512), dtype=np.uint64)
    _set_bits(l2_mask, l2_of_l1, (l1_key & 32767))
    leaf_tile = np.zeros(leaf_key.size, dtype=bool)
    tile_value = np.zeros(0, dtype=np.float32)
    l1_tile_mask = np.zeros((l1_key.size, 64), dtype=np.uint64)
    if tile_tol is not None and leaf_key.size:
        cnt = np.diff(np.append(leaf_first, n))
        tiles = []
        for lf in np.nonzero(cnt == 512)[0]:
            v = val[leaf_first[lf]:leaf_first[lf] + 512]
            mn, mx = np.float32(v.min()), np.float32(v.max())   # NaN propagates: never a tile
            if np.float32(mx - mn) <= np.float32(tile_tol):
                leaf_tile[lf] = True
                tiles.append(np.float32(np.float32(mn + mx) * np.float32(0.5)))
        tile_value = np.array(tiles, dtype=np.float32)
        if tile_value.size:
            val = val.copy()
            for t, lf in enumerate(np.nonzero(leaf_tile)[0]):
                val[leaf_first[lf]:leaf_first[lf] + 512] = tile_value[t]
            _set_bits(l1_tile_mask, l1_of_leaf[leaf_tile], (leaf_key[leaf_tile] & 4095))
    return dict(
        leaf_tile=leaf_tile, tile_value=tile_value, l1_tile_mask=l1_tile_mask,
        n=n, ijk=ijk, val=val, key=key,
        leaf_origin=ijk[leaf_first] & ~7, leaf_mask=leaf_mask, leaf_l1=l1_of_leaf,
        leaf_first=leaf_first,
        l1_origin=ijk[l1_first] & ~127, l1_mask=l1_mask, l1_l2=l2_of_l1,
        l2_origin=ijk[l2_first] & ~4095, l2_mask=l2_mask,
    )


def mask_bits(words: np.ndarray) -> np.ndarray:
    """Expand mask words [rows, W] into booleans [rows, 64*W] (bit b = word b>>6, bit b&63)."""
    sh = np.arange(64, dtype=np.uint64)
    return ((words[:, :, None] >> sh) & np.uint64(1)).astype(bool).reshape(words.shape[0], -1)


def l1_origins_from_upper(l2_origin: np.ndarray, l2_mask: np.ndarray) -> np.ndarray:
    """Level-1 node origins from the level-2 child masks, in canonical order (Section 3.5)."""
    out = []
    bits = mask_bits(l2_mask)
    for n in range(l2_origin.shape[0]):
        slot = np.nonzero(bits[n])[0]
        rel = np.stack([slot >> 10, (slot >> 5) & 31, slot & 31], 1) * 128
        out.append(np.asarray(l2_origin[n], dtype=np.int64)[None] + rel)
    return np.concatenate(out).astype(np.int64) if out else np.zeros((0, 3), np.int64)


def domain(ijk: np.ndarray):
    """Normalisation domain of the encodings: origin (level-1 aligned) and power-of-two extent E >= 128."""
    ijk = np.asarray(ijk, dtype=np.int64)
    lo = (ijk.min(0) >> 7) << 7
    hi = ((ijk.max(0) >> 7) + 1) << 7
    ext = int((hi - lo).max())
    log2e = 7
    while (1 << log2e) < ext:
        log2e += 1
    return lo, log2e
