"""Explicit-grid samplers, isosurface points and the modified Chamfer distance in FP64 (test
infrastructure).

Samplers of the explicit VDB (Section 4.4 compares NeuralVDB with order-0, 1 and 3
samplers): inactive voxels take the background.  Order 0: the voxel nearest p,
floor(p + 1/2).  Order 1: trilinear over the corners of the cell floor(p), corner
c = 4a + 2b + d weighted (wx wy) wz with w = t or 1 - t.  Order 3: tricubic Catmull-Rom
over the 4 x 4 x 4 voxels floor(p) - 1 .. floor(p) + 2, per-axis weights of t (Catmull &
Rom 1974: the cubic through the two middle samples with slopes from their neighbours).
Isosurface points (Eq. 4): for every active voxel v and axis a with v + e_a active and of
the other sign (v < 0 versus v >= 0), the zero of the linear interpolant v + t e_a,
t = val(v) / (val(v) - val(v + e_a)).  mCD = 1/(2 N1) sum |SDF_2(v1)| + 1/(2 N2) sum
|SDF_1(v2)|, each SDF sampled trilinearly (reading of Eq. 4: the distances enter by
absolute value).
"""
from __future__ import annotations

import numpy as np

from . import vdb


class Lookup:
    """Value of arbitrary voxels of a grid (background where inactive)."""

    def __init__(self, grid: dict, background: float):
        keys = vdb.canonical_key(grid["ijk"])
        self.order = np.argsort(keys)
        self.keys = keys[self.order]
        self.val = grid["val"].astype(np.float64)[self.order]
        self.bg = background

    def __call__(self, ijk: np.ndarray) -> np.ndarray:
        ijk = np.asarray(ijk, np.int64)
        inside = np.all((ijk >= 0) & (ijk < vdb.COORD_LIMIT), axis=-1)
        k = vdb.canonical_key(np.where(inside[..., None], ijk, 0).reshape(-1, 3)).reshape(inside.shape)
        pos = np.clip(np.searchsorted(self.keys, k), 0, len(self.keys) - 1)
        hit = inside & (self.keys[pos] == k)
        return np.where(hit, self.val[pos], self.bg)


def catmull_rom(t: np.ndarray) -> np.ndarray:
    """Weights [N, 4] of the samples at offsets -1, 0, 1, 2."""
    t = np.asarray(t, np.float64)
    return np.stack([0.5 * (-t ** 3 + 2 * t ** 2 - t), 0.5 * (3 * t ** 3 - 5 * t ** 2 + 2),
                     0.5 * (-3 * t ** 3 + 4 * t ** 2 + t), 0.5 * (t ** 3 - t ** 2)], -1)


def sample(grid: dict, background: float, pts: np.ndarray, order: int) -> np.ndarray:
    look = Lookup(grid, background)
    p = np.asarray(pts, np.float64)
    if order == 0:
        return look(np.floor(p + 0.5).astype(np.int64))
    c0 = np.floor(p).astype(np.int64)
    t = p - c0
    out = np.zeros(len(p))
    if order == 1:
        for c in range(8):
            off = np.array([(c >> 2) & 1, (c >> 1) & 1, c & 1])
            w = np.ones(len(p))
            for d in range(3):
                w = w * (t[:, d] if off[d] else 1.0 - t[:, d])
            out += w * look(c0 + off)
        return out
    wx, wy, wz = (catmull_rom(t[:, d]) for d in range(3))
    for a in range(4):
        for b in range(4):
            for d in range(4):
                out += wx[:, a] * wy[:, b] * wz[:, d] * look(c0 + np.array([a - 1, b - 1, d - 1]))
    return out


def isosurface(grid: dict, background: float) -> np.ndarray:
    look = Lookup(grid, background)
    ijk = grid["ijk"].astype(np.int64)
    v0 = grid["val"].astype(np.float64)
    keys = vdb.canonical_key(ijk)
    pts = []
    for a in range(3):
        e = np.zeros(3, np.int64)
        e[a] = 1
        nb = ijk + e
        knb = vdb.canonical_key(nb)
        act = np.isin(knb, keys)
        v1 = look(nb)
        cross = act & ((v0 < 0) != (v1 < 0))
        t = v0 / np.where(cross, v0 - v1, 1.0)
        pts.append((np.nonzero(cross)[0], a, ijk + t[:, None] * e[None]))
    # canonical voxel order, then axis order
    rows = np.concatenate([np.stack([r, np.full(len(r), a)], -1) for r, a, _ in pts])
    coords = np.concatenate([p[r] for r, _, p in pts])
    order = np.lexsort((rows[:, 1], rows[:, 0]))
    return coords[order]


def mcd(ref: dict, rec: dict, background: float) -> float:
    v1, v2 = isosurface(ref, background), isosurface(rec, background)
    s2 = np.abs(sample(rec, background, v1, 1))
    s1 = np.abs(sample(ref, background, v2, 1))
    return float(s2.sum() / (2 * len(v1)) + s1.sum() / (2 * len(v2)))
