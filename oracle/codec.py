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

L1CLS, L0CLS, REG = 0, 1, 2
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
             subdomain=0, halo=8, resample=0, sampling=0)
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
    nets = [rng.xavier_net(opts["seed"], 3 * e + k, ffm[0] if k == 0 else ffm[1], opts["width"][k], opts["layers"][k])
            for e in range(n_exp) for k in range(3)]
    return dict(grid_class=grid_class, background=(half_width if grid_class == 0 else 0.0),
                half_width=half_width, origin=origin, log2_extent=log2e, ffm_size=list(ffm),
                width=list(opts["width"]), layers=list(opts["layers"]), q=[q1, q0], nets=nets,
                l2_origin=grid["l2_origin"], l2_mask=grid["l2_mask"], n_l2=grid["l2_origin"].shape[0],
                n_l1=grid["l1_origin"].shape[0], n_leaf=grid["leaf_origin"].shape[0], n_active=grid["n"],
                patches={}, moe=moe)


def level_coords(model: dict, net: int, ijk: np.ndarray) -> np.ndarray:
    """Network input coordinates: voxel units (level 0) or leaf units (level 1), relative to the origin."""
    c = np.asarray(ijk, dtype=np.int64) - model["origin"][None]
    return c >> 3 if net == L1CLS else c


def level_q(model: dict, net: int) -> np.ndarray:
    return model["q"][0] if net == L1CLS else model["q"][1]


def evaluate(model: dict, net: int, ijk: np.ndarray, chunk: int = 1 << 16) -> np.ndarray:
    """Raw network output at voxel coordinates (level-1 nets take leaf origins); with a
    domain decomposition, the gate-weighted average of the experts (oracle/moe.py)."""
    if model.get("moe") is not None:
        out = np.empty(len(ijk))
        for a in range(0, len(ijk), chunk):
            out[a:a + chunk] = MOE.evaluate(model, net, np.asarray(ijk)[a:a + chunk])
        return out
    out = np.empty(len(ijk))
    for a in range(0, len(ijk), chunk):
        z = N.encode(level_coords(model, net, ijk[a:a + chunk]), level_q(model, net))
        out[a:a + chunk] = N.forward(model["nets"][net], z)[0]
    return out


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
    if net == L1CLS:
        node, slot = idx >> 12, idx & 4095
        ijk = grid["l1_origin"][node] + 8 * _lattice16(slot)
        lab = vdb.test_bit(grid["l1_mask"], node, slot).astype(np.float64)
    elif net == L0CLS:
        leaf, off = idx >> 9, idx & 511
        ijk = grid["leaf_origin"][leaf] + _lattice8(off)
        lab = vdb.test_bit(grid["leaf_mask"], leaf, off).astype(np.float64)
    else:
        ijk = grid["ijk"][idx]
        v = grid["val"][idx].astype(np.float64)
        lab = v / model["half_width"] if model["grid_class"] == 0 else v
    return ijk, lab


def population_size(grid: dict, net: int) -> int:
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
    kind = N.LOSS_BCE if net != REG else opts["loss"]
    q = level_q(model, net)
    pop = None if moe is None else MOE.population(grid, model, expert, net)
    sampling = opts.get("sampling", SPARSE) if net == REG else SPARSE
    if sampling == BLOCKED:
        npop = grid["leaf_origin"].shape[0] * 512
    elif sampling == DENSE:
        npop = 1 << (3 * model["log2_extent"])
    else:
        npop = population_size(grid, net) if pop is None else len(pop)
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
    """Source embedding (Section 3.3.2): every candidate whose decision differs from the truth."""
    l1c = l1_candidates(grid["l1_origin"])
    pred1 = evaluate(model, L1CLS, l1c) > 0
    truth1 = vdb.mask_bits(grid["l1_mask"]).reshape(-1)
    l1_off, l1_idx = _csr(pred1 != truth1, grid["l1_origin"].shape[0], 4096)
    l0c = l0_candidates(grid["leaf_origin"])
    pred0 = evaluate(model, L0CLS, l0c) > 0
    truth0 = vdb.mask_bits(grid["leaf_mask"]).reshape(-1)
    l0_off, l0_idx = _csr(pred0 != truth0, grid["leaf_origin"].shape[0], 512)
    model["patches"][prec] = dict(l1_off=l1_off, l1_idx=l1_idx, l0_off=l0_off, l0_idx=l0_idx)
    return model["patches"][prec]


def _apply_patches(pred: np.ndarray, off: np.ndarray, idx: np.ndarray, per: int) -> np.ndarray:
    out = pred.copy().reshape(-1, per)
    for r in range(out.shape[0]):
        for b in idx[off[r]:off[r + 1]]:
            out[r, b] = not out[r, b]
    return out.reshape(-1)


def decode_topology(model: dict, prec: int = PREC_FP32):
    """Top-down topology decode: (level-1 origins, leaf origins, leaf active masks as bool [n_leaf, 512])."""
    p = model["patches"][prec]
    l1_origin = vdb.l1_origins_from_upper(model["l2_origin"], model["l2_mask"])
    l1c = l1_candidates(l1_origin)
    child = _apply_patches(evaluate(model, L1CLS, l1c) > 0, p["l1_off"], p["l1_idx"], 4096)
    leaf_origin = l1c[child]
    l0c = l0_candidates(leaf_origin)
    act = _apply_patches(evaluate(model, L0CLS, l0c) > 0, p["l0_off"], p["l0_idx"], 512)
    return l1_origin, leaf_origin, act.reshape(-1, 512)


def decompress(model: dict, prec: int = PREC_FP32):
    """Decoded voxels (ijk [n,3], values [n]) in canonical order."""
    _, leaf_origin, act = decode_topology(model, prec)
    ijk = l0_candidates(leaf_origin)[act.reshape(-1)]
    y = evaluate(model, REG, ijk)
    val = y * model["half_width"] if model["grid_class"] == 0 else y
    return ijk, val


def value_scale(model: dict) -> float:
    return model["half_width"] if model["grid_class"] == 0 else 1.0


def query(model: dict, pts: np.ndarray, active_keys: np.ndarray):
    """Trilinear point query on [Hash,5,4,NN(3)].

    active_keys: sorted canonical keys of the active voxels (the explicit topology).
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
        if act.any():
            val[act] = evaluate(model, REG, ijk[act]) * value_scale(model)
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
