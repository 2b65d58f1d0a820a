"""Active tiles, the ternary level-1 classifier, the tile value regressor and the sin
activation on the GPU against the FP64 oracle (Sections 3.1, 3.3.1, 3.5; the activation
appendix).

Tile pruning bit-exact (flags, masks, values); initial networks bit-exact; network outputs at
1e-5 of the head scale (FP32) and the tensor-core bar (tile regressor); the first Adam step
of every network on the same samples; the ternary decode restores the topology exactly with
every tile voxel carrying its regressed value; queries answer tile corners from the tiles;
blob round trip; sin models decoded at FP32 and on the 16-bit tensor-core modes, each kernel
held to its precision's stated arithmetic; FP8 and BF16 training of sin networks refused; the
ternary classifier's cross-entropy gradient at FP32 and on the BF16 tensor-core step, and
BF16 training of a whole ternary model.
"""
import numpy as np
import pytest
import torch

import paper_2208_04448_b300 as nv
from fixtures import tiled_fog, workload
from gpu_helpers import bf16_weight_sensitivity, tc_bar
from oracle import blob, codec, vdb
from oracle import nets as N

pytestmark = pytest.mark.gpu

SEED, SIGMA = 9, 1.0
SHAPE = dict(width=[32, 32, 32], layers=[2, 2, 2])


def _grid(tol=0.0, big=False):
    ijk, val = tiled_fog(96, 40, 40) if big else tiled_fog()
    ref = vdb.build(ijk, val, tol)
    g = nv.build(torch.from_numpy(ijk.astype(np.int32)).cuda(), torch.from_numpy(val).cuda(), 1, 0.0,
                 prune_tiles=True, tile_tolerance=tol)
    return ijk, val, ref, g


@pytest.mark.parametrize("tol", [0.0, 0.01])
def test_tile_pruning_bit_exact(tol):
    ijk, val, ref, g = _grid(tol, big=True)
    assert g.info()["n_tiles"] == int(ref["leaf_tile"].sum()) > 0
    t = g.tiles()
    assert np.array_equal(t["leaf_tile"], ref["leaf_tile"])
    assert np.array_equal(t["l1_tile_mask"], ref["l1_tile_mask"])
    r = g.read()
    assert np.array_equal(r["ijk"], ref["ijk"]) and np.array_equal(r["val"], ref["val"])
    g0 = nv.build(torch.from_numpy(ijk.astype(np.int32)).cuda(), torch.from_numpy(val).cuda(), 1, 0.0)
    assert g0.info()["n_tiles"] == 0 and not g0.tiles()["leaf_tile"].any()


def test_tile_pruning_with_a_nan():
    """A leaf holding a NaN value is not a constant region on either side."""
    ijk, val = tiled_fog()
    val = val.copy()
    val[3] = np.nan                                       # inside the first constant leaf
    ref = vdb.build(ijk, val, 0.0)
    g = nv.build(torch.from_numpy(ijk.astype(np.int32)).cuda(), torch.from_numpy(val).cuda(), 1, 0.0,
                 prune_tiles=True, tile_tolerance=0.0)
    assert np.array_equal(g.tiles()["leaf_tile"], ref["leaf_tile"]) and not ref["leaf_tile"][0]
    assert g.info()["n_tiles"] == int(ref["leaf_tile"].sum()) == 17


def _opts(**kw):
    return codec.default_opts(seed=SEED, sigma=SIGMA, **SHAPE, **kw)


def test_ternary_initial_networks():
    ijk, val, ref, g = _grid()
    m = nv.compress(g, seed=SEED, ffm_sigma=SIGMA, steps=0, patch_precs=1, **SHAPE)
    om = codec.init_model(ref, 1, 0.0, _opts())
    got = blob.read(m.export())
    assert got["ternary"] and got["n_tiles"] == om["n_tiles"] == 18 and len(got["nets"]) == 4
    assert np.array_equal(got["q"][0], om["q"][0]) and np.array_equal(got["q"][1], om["q"][1])
    for a, b in zip(got["nets"], om["nets"]):
        assert np.shape(a["wh"]) == np.shape(b["wh"])
        assert np.array_equal(N.flatten(a), N.flatten(b).astype(np.float32).astype(np.float64))


def _scale(net, z):
    _, (hs, _) = N.forward(net, z)
    wh = np.atleast_2d(net["wh"])
    return (np.abs(hs[-1][:, None, :] * wh[None]).sum(-1) + np.abs(np.atleast_1d(net["bh"]))[None]).max(1)


@pytest.mark.parametrize("act", [N.ACT_RELU, N.ACT_SIN])
def test_ternary_networks_match_oracle(act):
    ijk, val, ref, g = _grid()
    kw = dict(activation=act, omega=1.5) if act else {}
    m = nv.compress(g, seed=SEED, ffm_sigma=SIGMA, steps=30, batch=1024, patch_precs=1, **SHAPE, **kw)
    om = blob.read(m.export())
    r = np.random.default_rng(2)
    pts = (ijk[r.integers(0, len(ijk), 3000)]).astype(np.int32)
    for net in range(4):
        want = codec.evaluate(om, net, pts)
        z = N.encode(codec.level_coords(om, net, pts), codec.level_q(om, net))
        sc = _scale(om["nets"][net], z)
        got = nv.mlp_eval(m, net, torch.from_numpy(pts).cuda(), nv.FP32).cpu().numpy()
        err = np.abs(got - want) / np.maximum(sc, 1e-30)[:, None] if got.ndim == 2 else np.abs(got - want) / sc
        assert err.max() <= 1e-5, (net, err.max())
    # the ternary classifier (three logits) and the tile regressor on the tensor cores: against
    # the FP64 network at the bar, and against the arithmetic each precision states
    from oracle import quant
    precs = (nv.FP16, nv.BF16X3, nv.BF16) + ((nv.FP8_E4M3,) if act == N.ACT_RELU else ())
    for net in (0, 3):
        want = codec.evaluate(om, net, pts)
        z = N.encode(codec.level_coords(om, net, pts), codec.level_q(om, net))
        sc = np.maximum(_scale(om["nets"][net], z), 1.0)
        sc = sc[:, None] if net == 0 else sc
        for prec in precs:
            got = nv.mlp_eval(m, net, torch.from_numpy(pts).cuda(), prec).cpu().numpy()
            spec = quant.forward(om["nets"][net], z, prec, codec.level_q(om, net), om["log2_extent"] - 3)
            dev = np.abs(got - spec) / sc
            assert np.quantile(dev, 0.99) <= 2e-4 and dev.max() <= 0.2, (net, prec, dev.max())
            if prec != nv.FP8_E4M3:
                assert (np.abs(got - want) / sc).max() <= tc_bar(prec), (net, prec)
    if act == N.ACT_SIN:   # sin networks: 16-bit tensor-core modes, not FP8
        with pytest.raises(nv.NvdbError) as e:
            nv.mlp_eval(m, 2, torch.from_numpy(pts).cuda(), nv.FP8_E4M3)
        assert e.value.status == nv.ERR_UNSUPPORTED


@pytest.mark.parametrize("act", [N.ACT_RELU, N.ACT_SIN])
def test_first_adam_step_of_every_network(act):
    ijk, val, ref, g = _grid()
    kw = dict(activation=act, omega=1.5) if act else {}
    m = nv.compress(g, seed=SEED, ffm_sigma=SIGMA, steps=1, batch=2048, lr=1e-3, patch_precs=1, **SHAPE, **kw)
    opts = _opts(steps=1, batch=2048, lr=1e-3, act=act, omega=1.5 if act else 1.0)
    om = codec.init_model(ref, 1, 0.0, opts)
    theta0 = [N.flatten(n) for n in om["nets"]]
    got = blob.read(m.export())
    for net in range(4):
        ls = codec.train_net(ref, om, net, opts)
        assert abs(m.losses(net)[0] - ls[0]) <= 1e-5 * max(1.0, abs(ls[0])), (net, m.losses(net)[0], ls[0])
        dw_ref = N.flatten(om["nets"][net]) - theta0[net]
        dw_got = N.flatten(got["nets"][net]) - theta0[net]
        big = np.abs(dw_ref) > 0.999e-3
        assert big.sum() > 0
        assert np.abs(dw_got[big] - dw_ref[big]).max() <= 2e-6, net


# BF16 gradient bars of the one-output networks' parity tests: per block, the relative L2
# error at most BF16_GRAD_K times the relative change of the FP64 gradient under BF16
# weights, plus u as a floor
GRAD_TOL, BF16_GRAD_K, BF16_U, BF16_LOSS_TOL = 1e-4, 3.0, 2.0 ** -9, 1e-2


@pytest.mark.parametrize("n", [1000, 37965])
@pytest.mark.parametrize("prec", [nv.FP32, nv.BF16])
@pytest.mark.parametrize("width,layers,ffm", [(32, 2, 32), (64, 4, 64)])
def test_ternary_gradient_parity(width, layers, ffm, prec, n):
    """The ternary classifier's softmax cross-entropy gradient (Section 3.3.1) through
    nvdb_mlp_grad against the oracle's backward: FP32 at 1e-4 of the largest entry, the
    tensor-core BF16 step at the BF16 bars.  n = 37965: 297 tiles, ragged."""
    ijk, val, ref, g = _grid()
    m = nv.compress(g, seed=SEED, ffm_sigma=SIGMA, steps=0, patch_precs=1, width=[width, 32, 32],
                    layers=[layers, 2, 2], ffm_size=[ffm, 32])
    om = blob.read(m.export())
    r = np.random.default_rng(width + n)
    pts = ijk[r.integers(0, len(ijk), n)].astype(np.int32)
    cls = r.integers(0, 3, n)
    net = om["nets"][0]
    z = N.encode(codec.level_coords(om, 0, pts), codec.level_q(om, 0))
    y, cache = N.forward(net, z)
    lref, gy = N.loss_and_grad(y, cls, N.LOSS_CE)
    gref = N.flatten(N.backward(net, cache, gy))
    got, lgot = nv.mlp_grad(m, 0, torch.from_numpy(pts).cuda(), torch.from_numpy(cls.astype(np.float32)).cuda(),
                            nv.LOSS_CE, prec)
    got = got.cpu().numpy()
    assert got.size == gref.size
    if prec == nv.FP32:
        assert np.abs(got - gref).max() <= GRAD_TOL * np.abs(gref).max()
        assert abs(lgot - lref) <= 1e-5 * max(1.0, abs(lref))
        return
    assert abs(lgot - lref) <= BF16_LOSS_TOL * max(1.0, abs(lref))
    gsens = bf16_weight_sensitivity(net, z, lambda yb: N.loss_and_grad(yb, cls, N.LOSS_CE)[1])
    sizes = [x for W, b in zip(net["W"], net["b"]) for x in (np.size(W), np.size(b))] + [np.size(net["wh"]),
                                                                                       np.size(net["bh"])]
    o = 0
    for sz in sizes:   # blocks W_0, b_0, ..., W_{L-1}, b_{L-1}, w_h [3][W], b_h [3]
        a, b, c = got[o:o + sz], gref[o:o + sz], gsens[o:o + sz]
        nb = max(np.linalg.norm(b), 1e-30)
        sens = np.linalg.norm(c - b) / nb
        assert np.linalg.norm(a - b) / nb <= BF16_GRAD_K * sens + BF16_U, (o, sz, sens)
        o += sz
    assert o == got.size


@pytest.mark.parametrize("prec", [nv.FP32, nv.BF16])
def test_ternary_gradient_refusals(prec):
    """A target that is not a class fails the call; the ternary classifier takes only the
    cross-entropy, the other networks not it."""
    ijk, val, ref, g = _grid()
    m = nv.compress(g, seed=SEED, ffm_sigma=SIGMA, steps=0, patch_precs=1, **SHAPE)
    pts = torch.from_numpy(ijk[:300].astype(np.int32)).cuda()
    tgt = torch.zeros(300, device="cuda")
    tgt[17] = 0.5
    with pytest.raises(nv.NvdbError) as e:
        nv.mlp_grad(m, 0, pts, tgt, nv.LOSS_CE, prec)
    assert e.value.status == nv.ERR_INVALID_ARG
    tgt[17] = 2.0
    nv.mlp_grad(m, 0, pts, tgt, nv.LOSS_CE, prec)          # the status was cleared
    for net, loss in ((0, nv.LOSS_BCE), (2, nv.LOSS_CE)):
        with pytest.raises(nv.NvdbError) as e:
            nv.mlp_grad(m, net, pts, tgt, loss, prec)
        assert e.value.status == nv.ERR_INVALID_ARG


def test_ternary_bf16_training_tracks_fp32():
    """Every network of a ternary model (the softmax-CE classifier included) trained by the
    tensor-core BF16 step from the same weights and Philox batches as FP32 training: first
    losses within the BF16 forward bar, trained losses at the FP32 run's level, and the
    model decodes to the exact topology with its tiles."""
    ijk, val, ref, g = _grid(big=True)
    kw = dict(seed=SEED, ffm_sigma=SIGMA, steps=120, batch=4096, patch_precs=0b11011, **SHAPE)
    m32 = nv.compress(g, train_prec=nv.FP32, **kw)
    m16 = nv.compress(g, train_prec=nv.BF16, **kw)
    for k in range(4):
        a, b = m32.losses(k), m16.losses(k)
        assert len(a) == len(b) == 120
        assert abs(b[0] - a[0]) <= BF16_LOSS_TOL * max(1.0, a[0]), k
        assert b[-20:].mean() <= 1.25 * a[-20:].mean() + 1e-4, (k, b[-20:].mean(), a[-20:].mean())
    dijk, dval, cnt = nv.decompress(m16, nv.FP16)
    assert cnt == [ref["n"]] and np.array_equal(dijk.cpu().numpy(), ref["ijk"])


@pytest.fixture(scope="module")
def trained():
    ijk, val, ref, g = _grid(big=True)
    m = nv.compress(g, seed=SEED, ffm_sigma=SIGMA, steps=60, batch=4096, patch_precs=0b11011, **SHAPE)
    return ijk, val, ref, g, m, blob.read(m.export())


@pytest.mark.parametrize("prec", [nv.FP32, nv.FP16, nv.BF16X3, nv.BF16])
def test_ternary_decode(trained, prec):
    ijk, val, ref, g, m, om = trained
    dijk, dval, cnt = nv.decompress(m, prec)
    dijk, dval = dijk.cpu().numpy(), dval.cpu().numpy()
    assert cnt == [ref["n"]] and np.array_equal(dijk, ref["ijk"])           # topology exact, tiles expanded
    first, tiles = ref["leaf_first"], np.nonzero(ref["leaf_tile"])[0]
    in_tile = np.zeros(ref["n"], bool)
    for lf in tiles:
        in_tile[first[lf]:first[lf] + 512] = True
    want_t = codec.evaluate(om, 3, ref["leaf_origin"][tiles])
    for t, lf in enumerate(tiles):
        v = dval[first[lf]:first[lf] + 512]
        assert np.all(v == v[0])
    got_t = dval[first[tiles]]
    want_v = codec.evaluate(om, 2, dijk[~in_tile])
    if prec == nv.FP32:
        assert np.abs(got_t - want_t).max() <= 1e-5 * max(1.0, np.abs(want_t).max())
        assert np.abs(dval[~in_tile] - want_v).max() <= 1e-4
    else:
        assert np.abs(got_t - want_t).max() <= tc_bar(prec) * 2
        assert np.abs(dval[~in_tile] - want_v).max() <= tc_bar(prec) * 2
    # the oracle decodes the exported blob to the same topology
    if prec == nv.FP32:
        oijk, oval = codec.decompress(om, 0)
        assert np.array_equal(oijk, dijk)
        assert np.abs(oval - dval).max() <= 1e-4


def test_ternary_blob_roundtrip_and_query(trained):
    ijk, val, ref, g, m, om = trained
    m2 = nv.model_import(m.export())
    assert m2.export() == m.export()
    a, b = nv.decompress(m, nv.FP16), nv.decompress(m2, nv.FP16)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    r = np.random.default_rng(5)
    pts = (ref["ijk"][r.integers(0, ref["n"], 4000)] + r.uniform(-0.5, 1.0, (4000, 3))).astype(np.float32)
    out, act = nv.query(m, torch.from_numpy(pts).cuda(), nv.FP32, active=True)
    tile_keys = np.sort(vdb.canonical_key(ref["leaf_origin"][ref["leaf_tile"]]) >> 9)
    want, bits = codec.query(om, pts, np.sort(vdb.canonical_key(ref["ijk"])), tile_keys)
    assert np.array_equal(act.cpu().numpy(), bits)
    assert np.abs(out.cpu().numpy() - want).max() <= 1e-4


def test_ternary_plan_and_tensor_core_queries(trained):
    """A ternary model through a graph-captured decode plan (same bits as nvdb_decompress) and
    point queries at FP16 (regressed corners on the tensor cores, tile corners from the cached
    tile values) against the oracle at the tensor-core bar."""
    ijk, val, ref, g, m, om = trained
    plan = nv.decompress_plan([m], nv.FP16)
    plan.launch()
    plan.check()
    dijk, dval, _ = nv.decompress(m, nv.FP16)
    assert torch.equal(plan.ijk, dijk) and torch.equal(plan.val, dval)
    r = np.random.default_rng(9)
    pts = (ref["ijk"][r.integers(0, ref["n"], 3000)] + r.uniform(-0.5, 1.0, (3000, 3))).astype(np.float32)
    out, act = nv.query(m, torch.from_numpy(pts).cuda(), nv.FP16, active=True)
    tile_keys = np.sort(vdb.canonical_key(ref["leaf_origin"][ref["leaf_tile"]]) >> 9)
    want, bits = codec.query(om, pts, np.sort(vdb.canonical_key(ref["ijk"])), tile_keys)
    assert np.array_equal(act.cpu().numpy(), bits)
    assert np.abs(out.cpu().numpy() - want).max() <= tc_bar(nv.FP16)


@pytest.fixture(scope="module")
def sin_model():
    ijk, val, _ = workload("sphere32")
    ref = vdb.build(ijk.numpy(), val.numpy())
    g = nv.build(ijk.cuda().contiguous(), val.cuda().contiguous(), 0, 3.0)
    m = nv.compress(g, seed=3, ffm_sigma=1.25, steps=40, batch=2048, patch_precs=0b11011, activation=nv.ACT_SIN,
                    omega=2.0, **SHAPE)
    return ref, g, m, blob.read(m.export())


@pytest.mark.parametrize("prec", [nv.FP32, nv.FP16, nv.BF16, nv.BF16X3])
def test_sin_model_decodes(sin_model, prec):
    ref, g, m, om = sin_model
    assert om["act"] == N.ACT_SIN and om["omega"] == 2.0
    dijk, dval, _ = nv.decompress(m, prec)
    assert np.array_equal(dijk.cpu().numpy(), ref["ijk"])
    want = codec.evaluate(om, 2, ref["ijk"])
    err = np.abs(dval.cpu().numpy() / 3.0 - want)
    assert err.max() <= (1e-5 if prec == nv.FP32 else tc_bar(prec)), err.max()


@pytest.mark.parametrize("prec", [nv.FP16, nv.BF16, nv.BF16X3])
def test_sin_kernel_matches_its_precision(sin_model, prec):
    """The sin instantiation of the tensor-core kernel against the arithmetic its precision
    states (oracle/quant.py): 99 % of rows within 2e-4 of max(head scale, 1), all within 2e-3."""
    from oracle import quant
    ref, g, m, om = sin_model
    r = np.random.default_rng(prec)
    pts = ref["ijk"][r.integers(0, ref["n"], 4096)].astype(np.int32)
    for net in (1, 2):
        z = N.encode(codec.level_coords(om, net, pts), codec.level_q(om, net))
        want = quant.forward(om["nets"][net], z, prec)
        sc = np.maximum(_scale(om["nets"][net], z), 1.0)
        got = nv.mlp_eval(m, net, torch.from_numpy(pts).cuda(), prec).cpu().numpy()
        e = np.abs(got - want) / sc
        assert np.quantile(e, 0.99) <= 2e-4 and e.max() <= 2e-3, (net, np.quantile(e, 0.99), e.max())


def test_sin_options_refused(sin_model):
    ref, g, m, om = sin_model
    for bad in (dict(patch_precs=0b101), dict(patch_precs=1, train_prec=nv.BF16)):
        with pytest.raises(nv.NvdbError) as e:
            nv.compress(g, seed=3, steps=1, activation=nv.ACT_SIN, omega=2.0, **SHAPE, **bad)
        assert e.value.status == nv.ERR_UNSUPPORTED
