"""Pins of the oracle's training population and of one whole training step (CPU only).

codec.population() maps a sample index to (voxel coordinates, label or target) for each
network (Section 3.2.1: the regressor samples active voxels only; Section 3.3.1: the
level-1 classifier labels leaf slots of level-1 nodes by the child mask, the level-0
classifier labels the voxels of every leaf by the active mask; Section 3.2: level-set
targets are the distances scaled to [-1, 1], fog targets the densities).  Every
expectation here is enumerated by brute force from the input voxel set, never from the
oracle's own masks, so a wrong slot-to-coordinate map, a label read from the wrong bit or
a target not divided by the half-width fails.  codec.train_net() is pinned by one Adam
step on a three-sample batch, with the gradient taken by central finite differences of a
loss written out sample by sample, and the first Adam step in its closed form
theta_1 = theta_0 - lr g / (|g| + eps).
"""
import math

import numpy as np
import pytest

from fixtures import workload
from oracle import codec, rng, vdb
from oracle import nets as N


def _voxels(name):
    ijk, val, _ = workload(name)
    return ijk.numpy().astype(np.int64), val.numpy()


@pytest.fixture(scope="module", params=["sphere32", "union128", "fog64"])
def case(request):
    ijk, val = _voxels(request.param)
    g = vdb.build(ijk, val)
    grid_class = 1 if request.param.startswith("fog") else 0
    half = 3.0
    m = codec.init_model(g, grid_class, half, codec.default_opts(width=[8, 8, 8], layers=[1, 1, 1]))
    truth = {tuple(c): float(v) for c, v in zip(ijk.tolist(), val.tolist())}
    return g, m, truth, grid_class, half


def _l1_slot_origin(node_origin, slot):
    # the 16^3 leaf slots of a level-1 node in x-major order, each 8 voxels apart
    n = 0
    for x in range(16):
        for y in range(16):
            for z in range(16):
                if n == slot:
                    return (node_origin[0] + 8 * x, node_origin[1] + 8 * y, node_origin[2] + 8 * z)
                n += 1
    raise AssertionError


def test_level1_population_brute_force(case):
    g, m, truth, _, _ = case
    occupied_leaves = {(i - i % 8, j - j % 8, k - k % 8) for (i, j, k) in truth}
    npop = codec.population_size(g, codec.L1CLS)
    assert npop == 4096 * len({(i - i % 128, j - j % 128, k - k % 128) for (i, j, k) in truth})
    idx = np.unique(np.concatenate([np.arange(0, npop, 97), rng.sample_indices(7, 0, 1, 512, npop)]))
    ijk, lab = codec.population(g, m, codec.L1CLS, idx)
    for t, (c, y) in enumerate(zip(ijk.tolist(), lab.tolist())):
        node, slot = int(idx[t]) // 4096, int(idx[t]) % 4096
        want = _l1_slot_origin(g["l1_origin"][node].tolist(), slot)
        assert tuple(c) == want
        assert y == (1.0 if want in occupied_leaves else 0.0)
    # every level-1 node origin is the 128-aligned corner of some input voxel
    assert {tuple(o) for o in g["l1_origin"].tolist()} == {(i - i % 128, j - j % 128, k - k % 128) for (i, j, k) in truth}


def test_level0_population_brute_force(case):
    g, m, truth, _, _ = case
    npop = codec.population_size(g, codec.L0CLS)
    assert npop == 512 * len({(i - i % 8, j - j % 8, k - k % 8) for (i, j, k) in truth})
    idx = np.unique(np.concatenate([np.arange(0, npop, 31), rng.sample_indices(7, 1, 1, 512, npop)]))
    ijk, lab = codec.population(g, m, codec.L0CLS, idx)
    for t, (c, y) in enumerate(zip(ijk.tolist(), lab.tolist())):
        leaf, off = int(idx[t]) // 512, int(idx[t]) % 512
        o = g["leaf_origin"][leaf].tolist()
        want = (o[0] + off // 64, o[1] + (off // 8) % 8, o[2] + off % 8)
        assert tuple(c) == want
        assert y == (1.0 if want in truth else 0.0)
    # the labels of the whole population count the input voxels exactly
    _, all_lab = codec.population(g, m, codec.L0CLS, np.arange(npop))
    assert int(all_lab.sum()) == len(truth)


def test_regressor_population_brute_force(case):
    g, m, truth, grid_class, half = case
    npop = codec.population_size(g, codec.REG)
    assert npop == len(truth)
    idx = np.unique(np.concatenate([np.arange(0, npop, 13), rng.sample_indices(7, 2, 1, 512, npop)]))
    ijk, tgt = codec.population(g, m, codec.REG, idx)
    for c, t in zip(ijk.tolist(), tgt.tolist()):
        v = truth[tuple(c)]
        assert t == (v / half if grid_class == 0 else v)
    if grid_class == 0:
        assert np.all(np.abs(tgt) < 1.0)   # band |d| < w maps into (-1, 1)


def _explicit_forward(p, q, c):
    """y for one coordinate, loops only: gamma, then ReLU layers, then the linear head."""
    m = q.shape[0]
    z = []
    for f in range(m):
        ph = sum(int(q[f, d]) * int(c[d]) for d in range(3)) % (1 << 32)
        if ph >= 1 << 31:
            ph -= 1 << 32
        z.append(ph)
    h = [math.cos(2 * math.pi * ph / 2 ** 32) for ph in z] + [math.sin(2 * math.pi * ph / 2 ** 32) for ph in z]
    for W, b in zip(p["W"], p["b"]):
        h = [max(0.0, sum(W[o][i] * h[i] for i in range(len(h))) + b[o]) for o in range(len(b))]
    return sum(p["wh"][i] * h[i] for i in range(len(h))) + p["bh"]


def _explicit_loss(theta, like, q, coords, targets, kind):
    p = N.unflatten(theta, like)
    total = 0.0
    for c, t in zip(coords, targets):
        y = _explicit_forward(p, q, c)
        if kind == N.LOSS_MSE:
            total += (y - t) ** 2
        else:   # BCE with logits
            total += max(y, 0.0) - y * t + math.log1p(math.exp(-abs(y)))
    return total / len(coords)


@pytest.mark.parametrize("net", [codec.L1CLS, codec.L0CLS, codec.REG])
def test_one_training_step_by_hand(net):
    ijk, val = _voxels("sphere32")
    g = vdb.build(ijk, val)
    truth = {tuple(c): float(v) for c, v in zip(ijk.tolist(), val.tolist())}
    opts = codec.default_opts(width=[4, 4, 4], layers=[2, 2, 2], ffm_size=[4, 4], sigma=1.0, seed=11,
                              steps=1, batch=3, lr=1e-2)
    m = codec.init_model(g, 0, 3.0, opts)
    r = np.random.default_rng(net)
    for p in m["nets"]:   # non-zero biases so that the bias gradients are exercised
        p["b"] = [r.standard_normal(b.shape) * 0.3 for b in p["b"]]
    like = m["nets"][net]
    theta0 = N.flatten(like).copy()
    # the three samples of step 1, mapped by brute force (not through codec.population)
    idx = rng.sample_indices(opts["seed"], net, 1, 3, codec.population_size(g, net))
    coords, targets = [], []
    for s in idx.tolist():
        if net == codec.L1CLS:
            o = _l1_slot_origin(g["l1_origin"][s // 4096].tolist(), s % 4096)
            occupied = {(i - i % 8, j - j % 8, k - k % 8) for (i, j, k) in truth}
            coords.append([(o[d] - int(m["origin"][d])) >> 3 for d in range(3)])
            targets.append(1.0 if o in occupied else 0.0)
        elif net == codec.L0CLS:
            lo = g["leaf_origin"][s // 512].tolist()
            v = (lo[0] + (s % 512) // 64, lo[1] + (s % 64) // 8, lo[2] + s % 8)
            coords.append([v[d] - int(m["origin"][d]) for d in range(3)])
            targets.append(1.0 if v in truth else 0.0)
        else:
            v = tuple(g["ijk"][s].tolist())
            coords.append([v[d] - int(m["origin"][d]) for d in range(3)])
            targets.append(truth[v] / 3.0)
    kind = N.LOSS_MSE if net == codec.REG else N.LOSS_BCE
    q = codec.level_q(m, net)
    loss0 = _explicit_loss(theta0, like, q, coords, targets, kind)
    grad = np.zeros_like(theta0)
    h = 1e-6
    for e in range(theta0.size):
        tp, tm = theta0.copy(), theta0.copy()
        tp[e] += h
        tm[e] -= h
        grad[e] = (_explicit_loss(tp, like, q, coords, targets, kind) - _explicit_loss(tm, like, q, coords, targets, kind)) / (2 * h)
    losses = codec.train_net(g, m, net, opts)
    assert losses[0] == pytest.approx(loss0, rel=1e-12, abs=1e-14)
    theta1 = N.flatten(m["nets"][net])
    step = theta1 - theta0
    want = -opts["lr"] * grad / (np.abs(grad) + N.ADAM_EPS)
    sure = np.abs(grad) > 1e-5            # finite differences resolve these gradients well
    assert sure.sum() >= 8
    assert np.allclose(step[sure], want[sure], rtol=1e-3, atol=1e-7)
    dead = np.abs(grad) < 1e-12           # units that no sample activates: no update at all
    assert np.all(step[dead] == 0.0)
    assert np.all(np.abs(step) <= opts["lr"] * (1 + 1e-12))
