"""Compress (train + patches), decompress and query -- the NeuralVDB codec in FP64.

[Hash,5,NN(4),NN(3)] (Section 3.3.1): the root and level-2 nodes stay
explicit; three networks replace the lower levels:
  net 0  level-1 mask classifier  input: leaf-index coordinates of the 16^3 child
         slots of every level-1 node; label: child mask c_1 (BCE; every voxel of
         the input is explicit, so there are no tiles and the ternary classifier
         reduces to child / no child)
  net 1  level-0 mask classifier  input: the 8^3 voxel coordinates of every leaf;
         label: active mask a_0 (BCE)
  net 2  voxel value regressor    input: active voxel coordinates only (Section
         3.2.1); target: value / half_width for level sets (range [-1, 1]),
         the value itself for fog (Section 3.2, after Eq. 1); MSE (Eq. 1) or L1.
With tiles (a grid built with tile pruning, oracle/vdb.py), net 0 is the ternary
level-1 classifier of Section 3.3.1: three logits per slot, classes 0 = child leaf,
1 = active tile, 2 = inactive tile, decided by the first maximum and trained with
cross-entropy over softmax; a fourth network, the tile value regressor (net 3), maps
the leaf-unit coordinate of each active tile to its value (target scaled as the
voxels'), and the level-0 networks train on the leaves that are not tiles.
Every network uses the model's activation (ReLU, or sin with frequency omega; oracle/nets.py).
Every misclassified candidate is stored as a patch (Section 3.3.2), both
false positives and false negatives, so that decoding restores the topology
exactly; the decision is logit > 0.
Decoding (Section 3.5, offline sequential access) runs top-down: level-1 node
origins from the level-2 child masks, level-1 classification + patches ->
leaves, level-0 classification + patches -> active voxels, regression ->
values.  Point queries (Section 3.5, online random access, [Hash,5,4,NN(3)])
look the 8 corners of the enclosing cell up in the explicit topology, regress
the active corners and blend trilinearly; inactive corners take the
background (+half_width for level sets, 0 for fog).
"""
from __future__ import annotations

import numpy as np

from . import moe as MOE
from . import nets as N
from . import rng, vdb

L1CLS, L0CLS, REG, TILE = 0, 1, 2, 3
CHILD, ACTIVE_TILE, INACTIVE = 0, 1, 2
PREC_FP32, PREC_BF16, PREC_FP8, PREC_FP16, PREC_BF16X3 = 0, 1, 2, 3, 4


def _lattice16(s):
    s = np.asarray(s, dtype=np.int64)
    return np.stack([s >> 8, (s >> 4) & 15, s & 15], -1)


def _lattice8(o):
    o = np.asarray(o, dtype=np.int64)
    return np.stack([o >> 6, (o >> 3) & 7, o & 7], -1)


def default_opts(**kw) -> dict:
    o = dict(width=[32, 32, 32], layers=[3, 3, 3], ffm_size=None, sigma=10.0, seed=1,
             steps=200, batch=4096, lr=1e-3, lr_decay=0.975, lr_interval=100, loss=N.LOSS_MSE,
             subdomain=0, halo=8, resample=0, sampling=0, act=N.ACT_RELU, omega=1.0,
             tile_width=None, tile_layers=None)
    o.update(kw)
    if o["ffm_size"] is None:
        o["ffm_size"] = [o["width"][0], max(o["width"][1], o["width"][2])]
    return o


def init_model(grid: dict, grid_class: int, half_width: float, opts: dict) -> dict:
    """Model with initial (untrained) networks and the grid's explicit upper tree."""
    origin, log2e = vdb.domain(grid["ijk"])
    E = 1 << log2e
    moe = MOE.plan(grid["ijk"], origin, log2e, opts["subdomain"], opts["halo"]) if opts.get("subdomain") else None
    if moe is not None:
        E = moe["size"]          # each expert normalises over its subdomain (Section 3.4)
    n_exp = 1 if moe is None else len(moe["origins"])
    ffm = opts["ffm_size"]
    q1 = rng.ffm_increments(opts["seed"], 1, ffm[0] // 2, opts["sigma"], E // 8)
    q0 = rng.ffm_increments(opts["seed"], 0, ffm[1] // 2, opts["sigma"], E)
    ternary = bool(np.any(grid.get("leaf_tile", np.zeros(0, bool))))
    if ternary and moe is not None:
        raise ValueError("active tiles with a domain decomposition are not supported")
    nets = [rng.xavier_net(opts["seed"], 3 * e + k, ffm[0] if k == 0 else ffm[1], opts["width"][k], opts["layers"][k],
                           3 if (ternary and k == L1CLS) else 1)
            for e in range(n_exp) for k in range(3)]
    tw = opts["tile_width"] or opts["width"][0]
    tl = opts["tile_layers"] or opts["layers"][0]
    if ternary:
        nets.append(rng.xavier_net(opts["seed"], TILE, ffm[0], tw, tl))
    for n in nets:
        n["act"], n["omega"] = opts["act"], float(np.float32(opts["omega"]))
    return dict(grid_class=grid_class, background=(half_width if grid_class == 0 else 0.0),
                half_width=half_width, origin=origin, log2_extent=log2e, ffm_size=list(ffm),
                width=list(opts["width"]), layers=list(opts["layers"]), q=[q1, q0], nets=nets,
                ternary=ternary, tile_shape=(tw, tl), act=opts["act"], omega=float(np.float32(opts["omega"])),
                n_tiles=int(np.sum(grid.get("leaf_tile", np.zeros(0, bool)))),
                l2_origin=grid["l2_origin"], l2_mask=grid["l2_mask"], n_l2=grid["l2_origin"].shape[0],
                n_l1=grid["l1_origin"].shape[0], n_leaf=grid["leaf_origin"].shape[0], n_active=grid["n"],
                patches={}, moe=moe)


def level_coords(model: dict, net: int, ijk: np.ndarray) -> np.ndarray:
    """Network input coordinates: voxel units (level 0) or leaf units (level 1), relative to the origin."""
    c = np.asarray(ijk, dtype=np.int64) - model["origin"][None]
    return c >> 3 if net in (L1CLS, TILE) else c


def level_q(model: dict, net: int) -> np.ndarray:
    return model["q"][0] if net in (L1CLS, TILE) else model["q"][1]


def evaluate(model: dict, net: int, ijk: np.ndarray, chunk: int = 1 << 16) -> np.ndarray:
    """Raw network output at voxel coordinates (level-1 nets take leaf origins); with a
    domain decomposition, the gate-weighted average of the experts (oracle/moe.py)."""
    if model.get("moe") is not None:
        out = np.empty(len(ijk))
        for a in range(0, len(ijk), chunk):
            out[a:a + chunk] = MOE.evaluate(model, net, np.asarray(ijk)[a:a + chunk])
        return out
    wide = np.ndim(model["nets"][net]["wh"]) == 2
    out = np.empty((len(ijk), 3) if wide else len(ijk))
    for a in range(0, len(ijk), chunk):
        z = N.encode(level_coords(model, net, ijk[a:a + chunk]), level_q(model, net))
        out[a:a + chunk] = N.forward(model["nets"][net], z)[0]
    return out


def nontile_leaves(grid: dict) -> np.ndarray:
    return np.nonzero(~grid.get("leaf_tile", np.zeros(grid["leaf_origin"].shape[0], bool)))[0]


def nontile_voxels(grid: dict) -> np.ndarray:
    """Indices (canonical order) of the voxels of the leaves that are not tiles."""
    lt = grid.get("leaf_tile", np.zeros(grid["leaf_origin"].shape[0], bool))
    first = np.append(grid["leaf_first"], grid["n"])
    keep = np.repeat(~lt, np.diff(first))
    return np.nonzero(keep)[0]


def l1_class(grid: dict, node, slot) -> np.ndarray:
    """Ternary level-1 label of slots: 0 child leaf, 1 active tile, 2 inactive."""
    child = vdb.test_bit(grid["l1_mask"], node, slot)
    tile = vdb.test_bit(grid["l1_tile_mask"], node, slot) if "l1_tile_mask" in grid else np.zeros_like(child)
    return np.where(tile, ACTIVE_TILE, np.where(child, CHILD, INACTIVE))


SPARSE, BLOCKED, DENSE = 0, 1, 2


def _voxel_target(grid: dict, model: dict, ijk: np.ndarray) -> np.ndarray:
    """Regressor target of arbitrary voxels: value (scaled) where active, else the background
    (+half_width for level sets, scaled to +1; 0 for fog)."""
    keys = vdb.canonical_key(grid["ijk"])
    order = np.argsort(keys)
    k = vdb.canonical_key(ijk)
    pos = np.clip(np.searchsorted(keys[order], k), 0, len(keys) - 1)
    hit = keys[order][pos] == k
    v = np.where(hit, grid["val"][order][pos].astype(np.float64), np.nan)
    if model["grid_class"] == 0:
        return np.where(hit, v / model["half_width"], 1.0)
    return np.where(hit, v, 0.0)


def regressor_population(grid: dict, model: dict, idx: np.ndarray, sampling: int):
    """Regressor samples of the sparsity ablation (Appendix C): SPARSE the active voxels
    (the method), BLOCKED every voxel of the leaves, DENSE every voxel of the domain's box."""
    if sampling == SPARSE:
        return population(grid, model, REG, idx)
    if sampling == BLOCKED:
        leaf, off = idx >> 9, idx & 511
        ijk = grid["leaf_origin"][leaf] + _lattice8(off)
    else:
        e = model["log2_extent"]
        ijk = model["origin"][None] + np.stack([idx >> (2 * e), (idx >> e) & ((1 << e) - 1), idx & ((1 << e) - 1)], -1)
    return ijk, _voxel_target(grid, model, ijk)


def population(grid: dict, model: dict, net: int, idx: np.ndarray):
    """Training population of a network: (voxel coordinates, label/target) for sample indices."""
    tern = model.get("ternary", False)
    if net == L1CLS:
        node, slot = idx >> 12, idx & 4095
        ijk = grid["l1_origin"][node] + 8 * _lattice16(slot)
        lab = l1_class(grid, node, slot) if tern else vdb.test_bit(grid["l1_mask"], node, slot).astype(np.float64)
    elif net == L0CLS:
        leaf, off = idx >> 9, idx & 511
        if tern:
            leaf = nontile_leaves(grid)[leaf]
        ijk = grid["leaf_origin"][leaf] + _lattice8(off)
        lab = vdb.test_bit(grid["leaf_mask"], leaf, off).astype(np.float64)
    elif net == TILE:
        ijk = grid["leaf_origin"][np.nonzero(grid["leaf_tile"])[0][idx]]
        v = grid["tile_value"][idx].astype(np.float64)
        lab = v / model["half_width"] if model["grid_class"] == 0 else v
    else:
        if tern:
            idx = nontile_voxels(grid)[idx]
        ijk = grid["ijk"][idx]
        v = grid["val"][idx].astype(np.float64)
        lab = v / model["half_width"] if model["grid_class"] == 0 else v
    return ijk, lab


def population_size(grid: dict, net: int, model: dict | None = None) -> int:
    if model is not None and model.get("ternary"):
        return [grid["l1_origin"].shape[0] * 4096, len(nontile_leaves(grid)) * 512, len(nontile_voxels(grid)),
                int(np.sum(grid["leaf_tile"]))][net]
    return [grid["l1_origin"].shape[0] * 4096, grid["leaf_origin"].shape[0] * 512, grid["n"]][net]


def train_net(grid: dict, model: dict, net: int, opts: dict, steps=None, log=None, expert: int = 0) -> list:
    """Sparse-field training of one network with Adam (Section 3.2, Section 3.2.1).  With a
    domain decomposition, `expert`'s network on its support's candidates (oracle/moe.py)."""
    moe = model.get("moe")
    slot = 3 * expert + net
    p = model["nets"][slot]
    theta = N.flatten(p)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    if net == L1CLS:
        kind = N.LOSS_CE if model.get("ternary") else N.LOSS_BCE
    else:
        kind = N.LOSS_BCE if net == L0CLS else opts["loss"]
    q = level_q(model, net)
    pop = None if moe is None else MOE.population(grid, model, expert, net)
    sampling = opts.get("sampling", SPARSE) if net == REG else SPARSE
    if sampling == BLOCKED:
        npop = grid["leaf_origin"].shape[0] * 512
    elif sampling == DENSE:
        npop = 1 << (3 * model["log2_extent"])
    else:
        npop = population_size(grid, net, model) if pop is None else len(pop)
    R = opts.get("resample", 0)
    losses = []
    for t in range(1, (opts["steps"] if steps is None else steps) + 1):
        if R:
            idx = rng.subset_indices(opts["seed"], slot, t, opts["batch"], R, npop)
        else:
            idx = rng.sample_indices(opts["seed"], slot, t, opts["batch"], npop)
        if sampling != SPARSE:
            ijk, lab = regressor_population(grid, model, idx, sampling)
        else:
            ijk, lab = population(grid, model, net, idx if pop is None else pop[idx])
        cur = N.unflatten(theta, p)
        c = level_coords(model, net, ijk) if moe is None else MOE.expert_coords(model, expert, net, ijk)
        y, cache = N.forward(cur, N.encode(c, q))
        loss, g = N.loss_and_grad(y, lab, kind)
        grads = N.backward(cur, cache, g)
        N.adam_step(theta, m, v, N.flatten(grads), t, N.lr_at(t, opts["lr"], opts["lr_decay"], opts["lr_interval"]))
        losses.append(loss)
        if log is not None:
            log(net, t, loss)
    model["nets"][slot] = N.unflatten(theta, p)
    return losses


def l1_candidates(l1_origin: np.ndarray) -> np.ndarray:
    """Leaf origins of all 16^3 slots of every level-1 node, node-major, slot order."""
    s = np.arange(4096)
    return (l1_origin[:, None, :] + 8 * _lattice16(s)[None]).reshape(-1, 3)


def l0_candidates(leaf_origin: np.ndarray) -> np.ndarray:
    o = np.arange(512)
    return (leaf_origin[:, None, :] + _lattice8(o)[None]).reshape(-1, 3)


def _csr(flags: np.ndarray, rows: int, per: int):
    f = flags.reshape(rows, per)
    cnt = f.sum(1)
    off = np.zeros(rows + 1, dtype=np.uint32)
    off[1:] = np.cumsum(cnt)
    idx = np.nonzero(f.reshape(-1))[0] % per
    return off, idx.astype(np.uint16)


def make_patches(grid: dict, model: dict, prec: int = PREC_FP32):
    """Source embedding (Section 3.3.2): every candidate whose decision differs from the truth.
    Ternary level 1: a patch is the slot with its true class in bits 12-13 (slot | class << 12);
    the level-0 lists cover every leaf of the grid, a tile's list empty (its voxels are all
    active without classification)."""
    l1c = l1_candidates(grid["l1_origin"])
    n1 = grid["l1_origin"].shape[0]
    if model.get("ternary"):
        pred = N.classify3(evaluate(model, L1CLS, l1c))
        node, slot = np.arange(n1 * 4096) >> 12, np.arange(n1 * 4096) & 4095
        truth = l1_class(grid, node, slot)
        l1_off, l1_idx = _csr(pred != truth, n1, 4096)
        bad = np.nonzero(pred != truth)[0]
        l1_idx = (l1_idx.astype(np.int64) | (truth[bad].astype(np.int64) << 12)).astype(np.uint16)
    else:
        pred1 = evaluate(model, L1CLS, l1c) > 0
        truth1 = vdb.mask_bits(grid["l1_mask"]).reshape(-1)
        l1_off, l1_idx = _csr(pred1 != truth1, n1, 4096)
    l0c = l0_candidates(grid["leaf_origin"])
    pred0 = evaluate(model, L0CLS, l0c) > 0
    truth0 = vdb.mask_bits(grid["leaf_mask"]).reshape(-1)
    diff0 = pred0 != truth0
    if model.get("ternary"):
        diff0 = diff0.reshape(-1, 512) & ~grid["leaf_tile"][:, None]
    l0_off, l0_idx = _csr(diff0, grid["leaf_origin"].shape[0], 512)
    model["patches"][prec] = dict(l1_off=l1_off, l1_idx=l1_idx, l0_off=l0_off, l0_idx=l0_idx)
    return model["patches"][prec]


def _apply_patches(pred: np.ndarray, off: np.ndarray, idx: np.ndarray, per: int) -> np.ndarray:
    out = pred.copy().reshape(-1, per)
    for r in range(out.shape[0]):
        for b in idx[off[r]:off[r + 1]]:
            out[r, b] = not out[r, b]
    return out.reshape(-1)


def _l1_classes(model: dict, p: dict, l1c: np.ndarray) -> np.ndarray:
    """Ternary level-1 classes of every slot after the patches (each patch sets its slot's class)."""
    cls = N.classify3(evaluate(model, L1CLS, l1c)).reshape(-1, 4096)
    for r in range(cls.shape[0]):
        for e in p["l1_idx"][p["l1_off"][r]:p["l1_off"][r + 1]]:
            cls[r, int(e) & 4095] = int(e) >> 12
    return cls.reshape(-1)


def decode_topology(model: dict, prec: int = PREC_FP32):
    """Top-down topology decode: (level-1 origins, leaf origins, leaf active masks as bool
    [n_leaf, 512], tile flag per leaf).  With tiles, the leaves are the slots classified as
    child leaf or active tile, in slot order; a tile's 512 voxels are all active."""
    p = model["patches"][prec]
    l1_origin = vdb.l1_origins_from_upper(model["l2_origin"], model["l2_mask"])
    l1c = l1_candidates(l1_origin)
    if model.get("ternary"):
        cls = _l1_classes(model, p, l1c)
        keep = cls <= ACTIVE_TILE
        tile = cls[keep] == ACTIVE_TILE
    else:
        keep = _apply_patches(evaluate(model, L1CLS, l1c) > 0, p["l1_off"], p["l1_idx"], 4096)
        tile = np.zeros(int(keep.sum()), bool)
    leaf_origin = l1c[keep]
    l0c = l0_candidates(leaf_origin)
    act = _apply_patches(evaluate(model, L0CLS, l0c) > 0, p["l0_off"], p["l0_idx"], 512).reshape(-1, 512)
    act[tile] = True
    return l1_origin, leaf_origin, act, tile


def decompress(model: dict, prec: int = PREC_FP32):
    """Decoded voxels (ijk [n,3], values [n]) in canonical order; a tile's voxels take the
    tile value regressed at the tile (net 3)."""
    _, leaf_origin, act, tile = decode_topology(model, prec)
    ijk = l0_candidates(leaf_origin)[act.reshape(-1)]
    in_tile = np.repeat(tile, act.sum(1))
    y = np.empty(len(ijk))
    y[~in_tile] = evaluate(model, REG, ijk[~in_tile])
    if tile.any():
        y[in_tile] = np.repeat(evaluate(model, TILE, leaf_origin[tile]), 512)
    val = y * model["half_width"] if model["grid_class"] == 0 else y
    return ijk, val


def value_scale(model: dict) -> float:
    return model["half_width"] if model["grid_class"] == 0 else 1.0


def query(model: dict, pts: np.ndarray, active_keys: np.ndarray, tile_keys: np.ndarray | None = None):
    """Trilinear point query on [Hash,5,4,NN(3)].

    active_keys: sorted canonical keys of the active voxels (the explicit topology);
    tile_keys: sorted leaf keys (canonical key >> 9) of the active tiles, whose voxels take
    the tile value regressed at the tile (net 3; Section 3.5: tiles answer from the tree).
    Corner c = a*4 + b*2 + d of cell floor(p) is floor(p) + (a, b, d); its weight is
    (wx * wy) * wz with w = t or 1 - t, t = p - floor(p); the result sums the corners in order.
    Returns (values [N], active corner bitmask uint8 [N]).
    """
    p = np.asarray(pts, dtype=np.float64)
    c0 = np.floor(p).astype(np.int64)
    t = p - c0
    out = np.zeros(p.shape[0])
    bits = np.zeros(p.shape[0], dtype=np.uint8)
    bg = model["background"]
    for corner in range(8):
        off = np.array([(corner >> 2) & 1, (corner >> 1) & 1, corner & 1])
        ijk = c0 + off[None]
        inside = np.all((ijk >= 0) & (ijk < vdb.COORD_LIMIT), axis=1)
        key = vdb.canonical_key(np.where(inside[:, None], ijk, 0))
        pos = np.searchsorted(active_keys, key)
        pos = np.minimum(pos, max(len(active_keys) - 1, 0))
        act = inside & (len(active_keys) > 0) & (active_keys[pos] == key if len(active_keys) else False)
        val = np.full(p.shape[0], bg)
        in_tile = np.zeros(p.shape[0], bool)
        if tile_keys is not None and len(tile_keys) and act.any():
            lk = key >> 9
            tp = np.minimum(np.searchsorted(tile_keys, lk), len(tile_keys) - 1)
            in_tile = act & (tile_keys[tp] == lk)
        reg = act & ~in_tile
        if reg.any():
            val[reg] = evaluate(model, REG, ijk[reg]) * value_scale(model)
        if in_tile.any():
            val[in_tile] = evaluate(model, TILE, ijk[in_tile] & ~7) * value_scale(model)
        wgt = np.ones(p.shape[0])
        for d in range(3):
            wgt = wgt * (t[:, d] if off[d] else 1.0 - t[:, d])
        out = out + wgt * val
        bits |= (act.astype(np.uint8) << corner)
    return out, bits


def iou_sdf(ref_val: np.ndarray, dec_val: np.ndarray) -> float:
    """IoU of the interiors {d < 0} over the (shared) active voxels (Section 4.1)."""
    a, b = ref_val < 0, dec_val < 0
    u = np.sum(a | b)
    return float(np.sum(a & b) / u) if u else 1.0


def rmse(ref_val: np.ndarray, dec_val: np.ndarray) -> float:
    return float(np.sqrt(np.mean((np.asarray(ref_val, np.float64) - dec_val) ** 2)))
