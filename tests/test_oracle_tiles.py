"""Pins of the oracle's tiles, ternary level-1 classifier, tile value regressor and sin
activation (CPU only; Sections 3.1, 3.3.1, 3.5 and the activation appendix).

Tile pruning is checked against a brute-force scan of the input voxel set; the softmax
cross-entropy against its closed form at equal logits; the three-output head and the sin
activation against central finite differences and a hand-expanded forward pass; the
ternary populations against enumeration from the input; and the ternary decode (patches
that set a slot's class) restores the source topology and tiles for untrained weights.
"""
import numpy as np
import pytest

from fixtures import tiled_fog
from oracle import blob, codec, rng, vdb
from oracle import nets as N


def _fog_with_tiles():
    return tiled_fog()


def test_tile_pruning_brute_force():
    ijk, val = _fog_with_tiles()
    for tol in (0.0, 0.01):
        gr = vdb.build(ijk, val, tol)
        vox = {tuple(c): float(x) for c, x in zip(ijk.tolist(), val.tolist())}
        leaves = {}
        for c, x in vox.items():
            leaves.setdefault((c[0] & ~7, c[1] & ~7, c[2] & ~7), []).append(np.float32(x))
        want = {}
        for o, xs in leaves.items():
            if len(xs) == 512 and np.float32(max(xs) - min(xs)) <= np.float32(tol):
                want[o] = np.float32((np.float32(min(xs)) + np.float32(max(xs))) * np.float32(0.5))
        got = {tuple(o): None for o in gr["leaf_origin"][gr["leaf_tile"]].tolist()}
        assert set(got) == set(want)
        assert np.array_equal(gr["tile_value"], np.array([want[o] for o in sorted(want, key=lambda o: vdb.canonical_key(np.array([o]))[0])], np.float32))
        assert (tol == 0.0 and len(want) == 18) or (tol == 0.01 and len(want) == 19)
        # a tile's voxels carry its value; the level-1 active mask marks the tile slots
        for t, lf in enumerate(np.nonzero(gr["leaf_tile"])[0]):
            f = gr["leaf_first"][lf]
            assert np.all(gr["val"][f:f + 512] == gr["tile_value"][t])
            o = gr["leaf_origin"][lf]
            slot = ((o[0] >> 3) & 15) << 8 | ((o[1] >> 3) & 15) << 4 | ((o[2] >> 3) & 15)
            assert vdb.test_bit(gr["l1_tile_mask"], gr["leaf_l1"][lf], slot)
        assert vdb.popcount(gr["l1_tile_mask"]) == len(want)
        assert np.array_equal(gr["ijk"], vdb.build(ijk, val)["ijk"])  # topology unchanged


def test_cross_entropy_closed_form_and_classes():
    y = np.zeros((4, 3))
    t = np.array([0, 1, 2, 1])
    l, g = N.loss_and_grad(y, t, N.LOSS_CE)
    assert abs(l - np.log(3.0)) < 1e-15
    want = np.full((4, 3), 1.0 / 3.0)
    want[np.arange(4), t] -= 1.0
    assert np.allclose(g, want / 4, atol=1e-16)
    # a confident correct logit: loss -> log(1 + 2 e^-d)
    l, _ = N.loss_and_grad(np.array([[10.0, 0.0, 0.0]]), np.array([0]), N.LOSS_CE)
    assert abs(l - np.log1p(2 * np.exp(-10.0))) < 1e-15
    assert N.classify3(np.array([[1.0, 1.0, 0.0], [0.0, 1.0, 1.0], [0.0, 0.0, 1.0], [2.0, 1.0, 2.0]])).tolist() == [0, 1, 2, 0]


def _tiny(act, n_out, seed=3):
    net = rng.xavier_net(seed, 0, 6, 5, 2, n_out)
    r = np.random.default_rng(seed)
    net["b"] = [r.normal(0, 0.3, 5) for _ in range(2)]
    net["bh"] = r.normal(0, 0.3, n_out) if n_out > 1 else 0.2
    net["act"], net["omega"] = act, 1.5
    return net


def test_sin_forward_hand_expanded():
    net = _tiny(N.ACT_SIN, 1)
    z = np.random.default_rng(0).normal(size=(3, 6))
    h1 = np.sin(1.5 * (z @ net["W"][0].T + net["b"][0]))
    h2 = np.sin(1.5 * (h1 @ net["W"][1].T + net["b"][1]))
    want = h2 @ net["wh"] + net["bh"]
    assert np.allclose(N.forward(net, z)[0], want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("act,n_out,kind", [(N.ACT_SIN, 1, N.LOSS_MSE), (N.ACT_SIN, 3, N.LOSS_CE),
                                            (N.ACT_RELU, 3, N.LOSS_CE)])
def test_backward_finite_differences(act, n_out, kind):
    net = _tiny(act, n_out)
    r = np.random.default_rng(7)
    z = r.normal(size=(9, 6))
    t = r.integers(0, 3, 9) if kind == N.LOSS_CE else r.normal(size=9)
    y, cache = N.forward(net, z)
    if act == N.ACT_RELU:   # probe away from the kinks
        assert min(np.abs(a).min() for a in cache[1]) > 1e-3
    _, g = N.loss_and_grad(y, t, kind)
    grad = N.flatten(N.backward(net, cache, g))
    theta = N.flatten(net)
    for e in range(theta.size):
        h = 1e-6 * max(1.0, abs(theta[e]))
        tp, tm = theta.copy(), theta.copy()
        tp[e] += h
        tm[e] -= h
        lp = N.loss_and_grad(N.forward(N.unflatten(tp, net), z)[0], t, kind)[0]
        lm = N.loss_and_grad(N.forward(N.unflatten(tm, net), z)[0], t, kind)[0]
        assert abs((lp - lm) / (2 * h) - grad[e]) <= 1e-6 * max(1.0, abs(grad[e])), e


def test_xavier_three_output_head_draw_order():
    a = rng.xavier_net(5, 0, 8, 4, 2, 1)
    b = rng.xavier_net(5, 0, 8, 4, 2, 3)
    for wa, wb in zip(a["W"], b["W"]):
        assert np.array_equal(wa, wb)                         # same hidden draws
    # head row 0 uses the same draws as the one-output head, bound sqrt(6/(w+3)) vs sqrt(6/(w+1))
    assert np.allclose(b["wh"][0], (a["wh"] * np.sqrt(5.0 / 7.0)).astype(np.float32), rtol=0, atol=1e-7)
    assert b["wh"].shape == (3, 4) and np.array_equal(b["bh"], np.zeros(3))


@pytest.fixture(scope="module")
def tiled():
    ijk, val = _fog_with_tiles()
    g = vdb.build(ijk, val, 0.0)
    opts = codec.default_opts(width=[32, 32, 32], layers=[2, 2, 2], seed=4, sigma=1.0, act=N.ACT_SIN, omega=1.5)
    m = codec.init_model(g, 1, 0.0, opts)
    return ijk, val, g, m, opts


def test_ternary_populations_brute_force(tiled):
    ijk, val, g, m, _ = tiled
    assert m["ternary"] and len(m["nets"]) == 4 and np.shape(m["nets"][0]["wh"]) == (3, 32)
    tiles = {tuple(o) for o in g["leaf_origin"][g["leaf_tile"]].tolist()}
    leaves = {tuple(o) for o in g["leaf_origin"].tolist()}
    idx = np.arange(g["l1_origin"].shape[0] * 4096)
    c, lab = codec.population(g, m, codec.L1CLS, idx)
    for o, y in zip(c.tolist(), lab.tolist()):
        o = tuple(o)
        assert y == (1 if o in tiles else 0 if o in leaves else 2)
    n0 = codec.population_size(g, codec.L0CLS, m)
    assert n0 == (len(leaves) - len(tiles)) * 512
    c, lab = codec.population(g, m, codec.L0CLS, np.arange(n0))
    act = {tuple(v) for v in ijk.tolist()}
    assert all(tuple(v[:3] & ~7) not in tiles for v in c) and np.array_equal(lab, [tuple(v) in act for v in c.tolist()])
    nr = codec.population_size(g, codec.REG, m)
    c, t = codec.population(g, m, codec.REG, np.arange(nr))
    vox = {tuple(a): float(b) for a, b in zip(ijk.tolist(), val.tolist())}
    assert nr == len(vox) - 512 * len(tiles) and all(t[i] == vox[tuple(c[i])] for i in range(0, nr, 37))
    c, t = codec.population(g, m, codec.TILE, np.arange(len(tiles)))
    assert {tuple(v) for v in c.tolist()} == tiles and np.all(t == 0.5)


def test_ternary_decode_restores_topology_and_tiles(tiled):
    ijk, val, g, m, _ = tiled
    codec.make_patches(g, m)
    p = m["patches"][0]
    assert np.all((p["l1_idx"] >> 12) <= 2)
    l1o, leafo, act, tile = codec.decode_topology(m)
    assert np.array_equal(leafo, g["leaf_origin"]) and np.array_equal(tile, g["leaf_tile"])
    assert np.array_equal(act, vdb.mask_bits(g["leaf_mask"]))
    dijk, dval = codec.decompress(m)
    assert np.array_equal(dijk, g["ijk"])
    first = g["leaf_first"]
    for lf in np.nonzero(g["leaf_tile"])[0]:
        v = dval[first[lf]:first[lf] + 512]
        assert np.all(v == v[0])                                       # one regressed value per tile
        assert abs(v[0] - codec.evaluate(m, codec.TILE, g["leaf_origin"][lf][None])[0]) <= 1e-12   # BLAS order


def test_ternary_blob_roundtrip(tiled):
    ijk, val, g, m, _ = tiled
    codec.make_patches(g, m)
    r = blob.read(blob.write(m))
    assert r["ternary"] and r["act"] == N.ACT_SIN and r["omega"] == m["omega"] and r["n_tiles"] == 18
    assert len(r["nets"]) == 4
    for a, b in zip(r["nets"], m["nets"]):
        assert np.array_equal(N.flatten(a), N.flatten(b).astype(np.float32).astype(np.float64))
    assert np.array_equal(r["patches"][0]["l1_idx"], m["patches"][0]["l1_idx"])


def test_ternary_first_adam_step(tiled):
    """One step of the ternary classifier: the same batch through forward, CE and the FD-pinned
    backward, then Adam's first step -lr g / (|g| + eps)."""
    ijk, val, g, m, opts = tiled
    o = dict(opts, steps=1, batch=64, lr=1e-3)
    mm = codec.init_model(g, 1, 0.0, o)
    theta0 = N.flatten(mm["nets"][0])
    idx = rng.sample_indices(o["seed"], 0, 1, 64, codec.population_size(g, 0, mm))
    c, lab = codec.population(g, mm, 0, idx)
    y, cache = N.forward(mm["nets"][0], N.encode(codec.level_coords(mm, 0, c), codec.level_q(mm, 0)))
    l, gy = N.loss_and_grad(y, lab, N.LOSS_CE)
    gr = N.flatten(N.backward(mm["nets"][0], cache, gy))
    ls = codec.train_net(g, mm, 0, o)
    assert abs(ls[0] - l) < 1e-15
    assert np.allclose(N.flatten(mm["nets"][0]) - theta0, -1e-3 * gr / (np.abs(gr) + 1e-8), rtol=0, atol=1e-15)
