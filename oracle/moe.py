"""Sparse domain decomposition (Section 3.4, Eq. 3) in FP64 (test infrastructure).

The domain is cut into a regular grid of cubic subdomains of size S voxels (a multiple of
512, Appendix E), anchored at the model's 128-aligned domain origin D; subdomains holding
no input voxel are discarded.  Every kept subdomain k (origin a_k = D + S i_k) has its own
expert: the three networks of the codec, with coordinates normalised over the subdomain
(x = (c - a_k) / S, Section 3.4), so the level's Fourier matrix is drawn for extent S
(S / 8 in the level-1 classifier's leaf units).

Gate (the paper's clamped tent, not learned): per axis, expert k covers its subdomain and a
halo of h voxels on each side (h = 8); the tent rises linearly across [a - h, a + h),
is 1 in the core and falls across [a + S - h, a + S + h).  Sampled at the centre of cell c
(integer coordinate c + 1/2):

    g(c; a) = min(clamp((c - a + h + 1/2) / (2h), 0, 1), clamp((a + S + h - 1/2 - c) / (2h), 0, 1))
    G_k(c)  = g(c_x; a_x) g(c_y; a_y) g(c_z; a_z).

Neighbouring tents cross so that their sum is 1 across the overlap (a partition of unity
on a full grid of subdomains); the values are multiples of 1/(4h), exact in binary.  At
most two subdomains per axis have g > 0 at a cell, so at most eight experts per point.
The output (Eq. 3, normalised as the paper's gate-weighted average) is

    y(c) = sum_k G_k(c) E_k(c) / sum_k G_k(c)

over the kept experts with G_k(c) > 0; only those are evaluated.  It applies to every
network: logits of the two classifiers (the decision stays logit > 0) and the regressor's
values.  The level-1 classifier works in leaf units (c = ijk >> 3, a / 8, S / 8, h / 8).

Training: each expert's networks are trained independently (the paper trains subdomains
concurrently on separate GPUs) on the candidates inside the expert's support, i.e. its
subdomain plus halo: level-1 slots whose leaf lies in it, the voxels of the leaves inside
it (the support is leaf-aligned since S and h are multiples of 8), and the active voxels
inside it.  Expert k's network j draws its initial weights and its sample stream with
network index 3k + j (k = 0 is the undecomposed model's stream).
"""
from __future__ import annotations

import numpy as np

from . import nets as N
from . import rng


def plan(ijk: np.ndarray, origin: np.ndarray, log2_extent: int, size: int, halo: int = 8) -> dict:
    """Subdomain grid over the domain [origin, origin + 2^log2_extent)^3; kept subdomains in
    lexicographic (x, y, z) order of their grid index."""
    if size <= 0 or size % 512:
        raise ValueError("subdomain size must be a positive multiple of 512")
    if halo <= 0 or halo % 8 or 2 * halo > size:
        raise ValueError("halo must be a positive multiple of 8 and at most size / 2")
    E = 1 << log2_extent
    n = -(-E // size)
    dims = (n, n, n)
    idx = (np.asarray(ijk, np.int64) - np.asarray(origin, np.int64)[None]) // size
    flat = np.unique((idx[:, 0] * n + idx[:, 1]) * n + idx[:, 2])
    expert_of = np.full(n * n * n, -1, dtype=np.int32)
    expert_of[flat] = np.arange(len(flat), dtype=np.int32)
    grid_idx = np.stack([flat // (n * n), (flat // n) % n, flat % n], -1)
    origins = np.asarray(origin, np.int64)[None] + size * grid_idx
    return dict(size=size, halo=halo, dims=dims, expert_of=expert_of, origins=origins.astype(np.int64))


def gate_axis(c, a, size: int, halo: int):
    """g(c; a) of the definition above (c, a broadcastable, level units)."""
    c = np.asarray(c, np.float64)
    a = np.asarray(a, np.float64)
    rise = np.clip((c - a + halo + 0.5) / (2 * halo), 0.0, 1.0)
    fall = np.clip((a + size + halo - 0.5 - c) / (2 * halo), 0.0, 1.0)
    return np.minimum(rise, fall)


def level_params(moe: dict, origin, net: int):
    """(domain origin, S, h) in the units of network `net` (leaves for the level-1 classifier)."""
    sh = 3 if net == 0 else 0
    return np.asarray(origin, np.int64) >> sh, moe["size"] >> sh, moe["halo"] >> sh


def experts_at(model: dict, net: int, ijk: np.ndarray):
    """Experts with G > 0 at every point: (ids [N, 8], gates [N, 8]); unused slots id -1, G 0.
    Slots are ordered by ascending expert id."""
    moe = model["moe"]
    D, S, h = level_params(moe, model["origin"], net)
    c = np.asarray(ijk, np.int64) >> (3 if net == 0 else 0)
    rel = c - D[None]
    base = rel // S
    n = moe["dims"][0]
    ids = np.full((len(c), 8), -1, dtype=np.int64)
    gs = np.zeros((len(c), 8))
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                gi = base + np.array([dx, dy, dz])[None]
                inside = np.all((gi >= 0) & (gi < n), axis=1)
                flat = np.where(inside, (gi[:, 0] * n + gi[:, 1]) * n + gi[:, 2], 0)
                e = np.where(inside, moe["expert_of"][flat], -1)
                a = D[None] + S * gi
                g = np.ones(len(c))
                for d in range(3):
                    g = g * gate_axis(c[:, d], a[:, d], S, h)
                use = (e >= 0) & (g > 0)
                if not use.any():
                    continue
                # place into the first free slot of each point
                free = np.argmax(ids < 0, axis=1)
                rows = np.nonzero(use)[0]
                ids[rows, free[rows]] = e[rows]
                gs[rows, free[rows]] = g[rows]
    order = np.argsort(np.where(ids < 0, np.iinfo(np.int64).max, ids), axis=1, kind="stable")
    ids = np.take_along_axis(ids, order, 1)
    gs = np.take_along_axis(gs, order, 1)
    return ids, gs


def expert_coords(model: dict, k: int, net: int, ijk: np.ndarray) -> np.ndarray:
    """Encoding coordinates of expert k (level units, relative to its subdomain origin)."""
    c = np.asarray(ijk, np.int64) - model["moe"]["origins"][k][None]
    return c >> 3 if net == 0 else c


def evaluate(model: dict, net: int, ijk: np.ndarray) -> np.ndarray:
    """Eq. 3: gate-weighted average of the experts with G > 0, each evaluated in FP64."""
    q = model["q"][0] if net == 0 else model["q"][1]
    ids, gs = experts_at(model, net, ijk)
    num = np.zeros(len(ijk))
    den = np.zeros(len(ijk))
    for k in np.unique(ids[ids >= 0]):
        rows, slots = np.nonzero(ids == k)
        z = N.encode(expert_coords(model, int(k), net, np.asarray(ijk)[rows]), q)
        y, _ = N.forward(model["nets"][3 * int(k) + net], z)
        num[rows] += gs[rows, slots] * y
        den[rows] += gs[rows, slots]
    if np.any(den <= 0):
        raise ValueError("a point outside every kept expert's support")
    return num / den


def support_box(model: dict, k: int, net: int):
    """Expert k's support [lo, hi) per axis in the level's units."""
    D, S, h = level_params(model["moe"], model["origin"], net)
    a = model["moe"]["origins"][k] >> (3 if net == 0 else 0)
    return a - h, a + S + h


def population(grid: dict, model: dict, k: int, net: int) -> np.ndarray:
    """Candidate indices of expert k's training population, in the undecomposed population's
    numbering (level-1: node * 4096 + slot; level-0: leaf * 512 + offset; regressor: voxel)."""
    lo, hi = support_box(model, k, net)
    if net == 0:
        s = np.arange(4096)
        lat = np.stack([s >> 8, (s >> 4) & 15, s & 15], -1)
        leaf = (grid["l1_origin"][:, None, :] >> 3) + lat[None]
        inside = np.all((leaf >= lo) & (leaf < hi), axis=2).reshape(-1)
        return np.nonzero(inside)[0].astype(np.int64)
    if net == 1:
        lo_o = grid["leaf_origin"]
        inside = np.all((lo_o >= lo) & (lo_o + 8 <= hi), axis=1)
        leaves = np.nonzero(inside)[0].astype(np.int64)
        return (leaves[:, None] * 512 + np.arange(512)[None]).reshape(-1)
    inside = np.all((grid["ijk"] >= lo) & (grid["ijk"] < hi), axis=1)
    return np.nonzero(inside)[0].astype(np.int64)
