"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (tolerances written per test): bit-exact for the tree build, the initial
parameters, topology, compacted lists and patch-corrected masks; 1e-5
relative (normalised by the head's dot-product scale) for FP32 network values;
1e-4 relative for FP32 gradients; 2e-2 of the band half-width for the
tensor-core precisions FP16, BF16 and compensated BF16 (gpu_helpers.TC_BARS); FP8 is
checked against the arithmetic it states in test_gpu_precision.py.
"""
import numpy as np
import pytest
import torch

import paper_2208_04448_b300 as nv
from fixtures import query_points, workload
from gpu_helpers import bf16_weight_sensitivity, oracle_forward_scale, randomise_biases, rel_err, round_bf16, tc_bar, tc_check
from oracle import blob, codec, vdb
from oracle import nets as N

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
GRAD_TOL = 1e-4
# BF16 training arithmetic rounds each operand of the forward, delta and weight-gradient
# products once to BF16 (unit roundoff u = 2^-9).  How much a gradient moves under
# such roundings depends on the network and the loss (sign-based L1 gradients move
# most), so the bar is relative to a measured sensitivity: per parameter block, the
# relative L2 error may be at most BF16_GRAD_K times the relative change of the FP64
# gradient when only the weights are rounded to BF16 (the kernel rounds weights,
# activations and deltas: a few roundings of the same size), plus u as a floor.
BF16_GRAD_K = 3.0
BF16_U = 2.0 ** -9
BF16_LOSS_TOL = 1e-2


def _cuda(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def _corner_sphere():
    a = np.arange(4084, 4109)
    g = np.stack(np.meshgrid(a, a, a, indexing="ij"), -1).reshape(-1, 3)
    d = np.sqrt(((g - 4096.5) ** 2).sum(1)) - 7.0
    sel = np.abs(d) < 3.0
    return g[sel].astype(np.int32), d[sel].astype(np.float32)


def _volume(name):
    if name == "corner":
        return _corner_sphere()
    ijk, val, _ = workload(name)
    return ijk.numpy(), val.numpy()


@pytest.fixture(scope="module")
def sphere128():
    ijk, val = _volume("sphere128")
    perm = np.random.default_rng(0).permutation(len(val))
    ijk, val = ijk[perm], val[perm]
    return ijk, val, vdb.build(ijk, val)


def _grid(ijk, val):
    return nv.build(_cuda(ijk, torch.int32), _cuda(val, torch.float32), 0, 3.0)


# ---------------------------------------------------------------------------- build (bit-exact)

@pytest.mark.parametrize("name", ["sphere32", "union128", "corner"])
def test_build_bit_exact(name):
    ijk, val = _volume(name)
    perm = np.random.default_rng(1).permutation(len(val))
    ijk, val = ijk[perm], val[perm]
    ref = vdb.build(ijk, val)
    g = _grid(ijk, val)
    got = g.read()
    assert np.array_equal(got["ijk"], ref["ijk"]) and np.array_equal(got["val"], ref["val"])
    assert np.array_equal(got["leaf_origin"], ref["leaf_origin"]) and np.array_equal(got["leaf_mask"], ref["leaf_mask"])
    assert np.array_equal(got["l1_origin"], ref["l1_origin"]) and np.array_equal(got["l1_mask"], ref["l1_mask"])
    info = g.info()
    o, l2e = vdb.domain(ijk)
    assert info["origin"] == list(o) and info["log2_extent"] == l2e and info["n_l2"] == ref["l2_origin"].shape[0]


def test_build_errors_and_empty():
    ijk = _cuda(np.array([[1, 2, 3], [4, 5, 6], [1, 2, 3]]), torch.int32)
    with pytest.raises(nv.NvdbError) as e:
        nv.build(ijk, _cuda(np.zeros(3), torch.float32))
    assert e.value.status == 2
    with pytest.raises(nv.NvdbError) as e:
        nv.build(_cuda(np.array([[1 << 21, 0, 0]]), torch.int32), _cuda(np.zeros(1), torch.float32))
    assert e.value.status == 1
    g = nv.build(torch.zeros((0, 3), dtype=torch.int32, device="cuda"), torch.zeros(0, device="cuda"))
    assert g.info()["n_leaf"] == 0


@pytest.mark.parametrize("case", ["one_voxel", "corners", "one_full_leaf"])
def test_tiny_and_extreme_grids_round_trip(case):
    """Degenerate grids through compress and decompress at every precision: one voxel; two
    voxels at opposite corners of the coordinate range (two level-2 nodes, extent 2^21); one
    full leaf.  Topology and order exact; values at the oracle's bars."""
    if case == "one_voxel":
        ijk, val = np.array([[5, 9, 300]]), np.array([0.5])
    elif case == "corners":
        ijk, val = np.array([[0, 0, 0], [(1 << 21) - 1] * 3]), np.array([-1.0, 2.0])
    else:
        a = np.arange(8)
        ijk = np.stack(np.meshgrid(a + 16, a + 8, a, indexing="ij"), -1).reshape(-1, 3)
        val = np.linspace(-2.5, 2.5, len(ijk))
    ijk, val = ijk.astype(np.int32), val.astype(np.float32)
    ref = vdb.build(ijk, val)
    m = nv.compress(_grid(ijk, val), seed=2, ffm_sigma=1.25, steps=5, batch=256, patch_precs=0b11111)
    om = blob.read(m.export())
    for prec in (0, 1, 2, 3, 4):
        dijk, dval, cnt = nv.decompress(m, prec)
        dijk, dval = dijk.cpu().numpy(), dval.cpu().numpy()
        assert cnt == [ref["n"]] and np.array_equal(dijk, ref["ijk"]), (case, prec)
        want, scale = oracle_forward_scale(om, 2, dijk)
        if prec == 0:
            assert rel_err(dval / 3.0, want, scale).max() <= FP32_TOL
        else:
            tc_check(prec, om, 2, dijk, dval / 3.0)


# ---------------------------------------------------------------------------- initial parameters (bit-exact)

def test_initial_parameters_bit_identical(sphere128):
    ijk, val, ref = sphere128
    m = nv.compress(_grid(ijk, val), steps=0, seed=123, ffm_sigma=1.25, width=[32, 32, 64], layers=[3, 2, 4],
                    patch_precs=1)
    got = blob.read(m.export())
    want = codec.init_model(ref, 0, 3.0, codec.default_opts(seed=123, sigma=1.25, width=[32, 32, 64], layers=[3, 2, 4]))
    assert np.array_equal(got["q"][0], want["q"][0]) and np.array_equal(got["q"][1], want["q"][1])
    for k in range(3):
        assert np.array_equal(N.flatten(got["nets"][k]), N.flatten(want["nets"][k]))
    assert list(got["origin"]) == list(want["origin"]) and got["log2_extent"] == want["log2_extent"]
    assert np.array_equal(got["l2_mask"], ref["l2_mask"])


# ---------------------------------------------------------------------------- network values

def _imported(ref, seed, width, layers, ffm=None):
    opts = codec.default_opts(seed=seed, sigma=1.25, width=width, layers=layers)
    if ffm:
        opts["ffm_size"] = ffm
    om = randomise_biases(codec.init_model(ref, 0, 3.0, opts), seed)
    codec.make_patches(ref, om)
    return om, nv.model_import(blob.write(om))


@pytest.mark.parametrize("shape", [([32, 32, 32], [3, 3, 3], None), ([32, 64, 64], [2, 4, 4], [32, 64]),
                                   ([64, 32, 64], [3, 3, 4], [64, 64])])
@pytest.mark.parametrize("prec", [0, 1, 3, 4])
def test_mlp_eval_parity(sphere128, shape, prec):
    ijk, val, ref = sphere128
    om, m = _imported(ref, 5, *shape)
    r = np.random.default_rng(2)
    pts = np.concatenate([ref["ijk"][r.integers(0, ref["n"], 1000)], r.integers(0, 128, (333, 3))]).astype(np.int32)
    for net in range(3):
        want, scale = oracle_forward_scale(om, net, pts)
        got = nv.mlp_eval(m, net, _cuda(pts, torch.int32), prec).cpu().numpy()
        if prec == 0:
            assert rel_err(got, want, scale).max() <= FP32_TOL
        else:
            assert (np.abs(got - want) / np.maximum(scale, 1.0)).max() <= tc_bar(prec)


# ---------------------------------------------------------------------------- gradients

@pytest.mark.parametrize("net,loss,n", [(0, 2, 1000), (1, 2, 1000), (2, 0, 1000), (2, 1, 1000), (2, 0, 37965)])
@pytest.mark.parametrize("prec", [0, 1])
def test_gradient_parity(sphere128, net, loss, n, prec):
    """n = 37965: 297 tiles (ragged), so blocks accumulate two or three tiles each."""
    ijk, val, ref = sphere128
    om, m = _imported(ref, 9, [32, 64, 64], [3, 4, 4], [32, 64])
    r = np.random.default_rng(net * 3 + loss)
    pts = ref["ijk"][r.integers(0, ref["n"], n)].astype(np.int32)
    tgt = (r.random(n) > 0.5).astype(np.float32) if loss == 2 else r.standard_normal(n).astype(np.float32)
    y, cache = N.forward(om["nets"][net], N.encode(codec.level_coords(om, net, pts), codec.level_q(om, net)))
    if loss == 1:   # keep L1 residuals away from zero so sign() is unambiguous
        tgt = (y + np.where(r.random(n) > 0.5, 0.3, -0.3)).astype(np.float32)
    lref, gy = N.loss_and_grad(y, tgt.astype(np.float64), loss)
    gref = N.flatten(N.backward(om["nets"][net], cache, gy))
    g, lgot = nv.mlp_grad(m, net, _cuda(pts, torch.int32), _cuda(tgt, torch.float32), loss, prec)
    g = g.cpu().numpy()
    if prec == 0:
        assert np.abs(g - gref).max() <= GRAD_TOL * np.abs(gref).max()
        assert abs(lgot - lref) <= 1e-5 * max(1.0, abs(lref))
    else:
        assert abs(lgot - lref) <= BF16_LOSS_TOL * max(1.0, abs(lref))
        p = om["nets"][net]
        gsens = bf16_weight_sensitivity(p, N.encode(codec.level_coords(om, net, pts), codec.level_q(om, net)),
                                        lambda yb: N.loss_and_grad(yb, tgt.astype(np.float64), loss)[1])
        sizes = [x for W, b in zip(p["W"], p["b"]) for x in (np.size(W), np.size(b))] + [np.size(p["wh"]), 1]
        o = 0
        for sz in sizes:   # blocks W_0, b_0, ..., W_{L-1}, b_{L-1}, w_h, b_h
            a, b, c = g[o:o + sz], gref[o:o + sz], gsens[o:o + sz]
            nb = max(np.linalg.norm(b), 1e-30)
            sens = np.linalg.norm(c - b) / nb
            assert np.linalg.norm(a - b) / nb <= BF16_GRAD_K * sens + BF16_U, (o, sz, sens)
            o += sz
        assert o == g.size


def test_gradient_precision_errors(sphere128):
    ijk, val, ref = sphere128
    om, m = _imported(ref, 9, [32, 64, 64], [3, 4, 4], [32, 64])
    pts = _cuda(ref["ijk"][:256], torch.int32)
    tgt = torch.zeros(256, device="cuda")
    for bad in (2, 3, 7):
        with pytest.raises(nv.NvdbError):
            nv.mlp_grad(m, 2, pts, tgt, 0, bad)


def test_first_adam_step_and_sample_stream(sphere128):
    ijk, val, ref = sphere128
    m = nv.compress(_grid(ijk, val), seed=77, ffm_sigma=1.25, steps=1, batch=4096, lr=1e-3, patch_precs=1)
    opts = codec.default_opts(seed=77, sigma=1.25, steps=1, batch=4096)
    om = codec.init_model(ref, 0, 3.0, opts)
    theta0 = [N.flatten(n) for n in om["nets"]]
    got = blob.read(m.export())
    for k in range(3):
        ls = codec.train_net(ref, om, k, opts)
        assert abs(m.losses(k)[0] - ls[0]) <= 1e-5 * max(1.0, abs(ls[0]))   # same Philox batch
        dw_ref = N.flatten(om["nets"][k]) - theta0[k]
        dw_got = N.flatten(got["nets"][k]) - theta0[k]
        big = np.abs(dw_ref) > 0.9e-3          # |g| >> eps: step = -lr sign(g)
        assert big.mean() > 0.5
        assert np.abs(dw_got[big] - dw_ref[big]).max() <= 2e-6


def test_training_trajectory_matches_oracle(sphere128):
    ijk, val, ref = sphere128
    m = nv.compress(_grid(ijk, val), seed=3, ffm_sigma=1.25, steps=200, batch=4096, patch_precs=1)
    opts = codec.default_opts(seed=3, sigma=1.25, steps=200, batch=4096)
    om = codec.init_model(ref, 0, 3.0, opts)
    for k in range(3):
        ls = np.array(codec.train_net(ref, om, k, opts))
        got = m.losses(k)
        assert abs(got[-20:].mean() - ls[-20:].mean()) <= 0.05 * ls[-20:].mean()
        assert abs(got[0] - ls[0]) <= 1e-5 * max(1.0, ls[0])


def test_bf16_training_tracks_fp32(sphere128):
    """Tensor-core (BF16) training from the same initial weights and Philox batches as FP32
    training: the first loss agrees within the BF16 forward bar, the trained loss reaches the
    FP32 run's level, and the trained model decodes with exact topology."""
    ijk, val, ref = sphere128
    g = _grid(ijk, val)
    kw = dict(seed=3, ffm_sigma=1.25, steps=200, batch=4096, patch_precs=0b11011, width=[32, 64, 64],
              layers=[3, 4, 4], ffm_size=[32, 64])
    m32 = nv.compress(g, train_prec=0, **kw)
    m16 = nv.compress(g, train_prec=1, **kw)
    for k in range(3):
        a, b = m32.losses(k), m16.losses(k)
        assert len(a) == len(b) == 200
        assert abs(b[0] - a[0]) <= BF16_LOSS_TOL * max(1.0, a[0])
        assert b[-20:].mean() <= 1.25 * a[-20:].mean() + 1e-4
    om = blob.read(m16.export())
    for k in range(3):   # the BF16 step stores BF16 weights and biases (the head stays FP32)
        net = om["nets"][k]
        for a in list(net["W"]) + list(net["b"]):
            assert np.array_equal(round_bf16(a), np.asarray(a, np.float64))
    want, scale = oracle_forward_scale(om, 2, ref["ijk"])
    for prec in (0, 1, 3, 4):   # BF16 decode of BF16 weights: two MMAs per K-step (no weight residual)
        dijk, dval, cnt = nv.decompress(m16, prec)
        assert cnt == [ref["n"]] and np.array_equal(dijk.cpu().numpy(), ref["ijk"])
        dv = dval.cpu().numpy()
        if prec == 0:
            assert rel_err(dv / 3.0, want, scale).max() <= FP32_TOL
        else:
            assert np.abs(dv - 3.0 * want).max() <= tc_bar(prec) * 3.0


def test_graph_replayed_training_equals_launched(sphere128):
    """Chunks of 50 training steps replay as a CUDA graph unless profiling is on (then every
    step is launched): 130 steps run a launched chunk, a replayed chunk and a launched
    remainder, and both ways give the same bits."""
    ijk, val, ref = sphere128
    g = _grid(ijk, val)
    kw = dict(seed=5, ffm_sigma=1.25, steps=130, batch=4096, patch_precs=1)
    for prec in (0, 1):
        nv.profile_enable(True)
        launched = nv.compress(g, train_prec=prec, **kw)
        nv.profile_enable(False)
        nv.profile_read()
        replayed = nv.compress(g, train_prec=prec, **kw)
        assert launched.export() == replayed.export()
        for k in range(3):
            assert np.array_equal(launched.losses(k), replayed.losses(k)) and len(replayed.losses(k)) == 130


def test_fused_adam_step_gives_the_same_bits(sphere128):
    """The BF16 step with Adam fused into its cooperative launch (grid barrier, then each CTA
    reduces a share of the partial slots in the same group order) against the two-launch step:
    identical model bytes and losses, over graph-replayed and launched chunks."""
    ijk, val, ref = sphere128
    g = _grid(ijk, val)
    kw = dict(seed=6, ffm_sigma=1.25, steps=120, batch=8192, patch_precs=1, train_prec=nv.BF16)
    try:
        nv.debug_inject(nv.INJECT_FUSED_ADAM, 1)
        fused = nv.compress(g, **kw)
    finally:
        nv.debug_inject(nv.INJECT_FUSED_ADAM, -1)
    split = nv.compress(g, **kw)
    assert fused.export() == split.export()
    for k in range(3):
        assert np.array_equal(fused.losses(k), split.losses(k))


def test_training_precision_errors(sphere128):
    ijk, val, ref = sphere128
    g = _grid(ijk, val)
    for bad in (2, 3):
        with pytest.raises(nv.NvdbError):
            nv.compress(g, train_prec=bad, steps=1)
    with pytest.raises(nv.NvdbError):   # the tensor-core step holds at most 4 hidden layers
        nv.compress(g, train_prec=1, steps=1, layers=[5, 3, 3])


# ---------------------------------------------------------------------------- decode

@pytest.mark.parametrize("name", ["sphere128", "union128", "corner"])
def test_decompress_parity(name):
    ijk, val = _volume(name)
    ref = vdb.build(ijk, val)
    m = nv.compress(_grid(ijk, val), seed=4, ffm_sigma=1.25, steps=50, batch=2048, width=[32, 64, 64],
                    layers=[3, 3, 4], patch_precs=0b11111)
    om = blob.read(m.export())
    for prec in (0, 1, 2, 3, 4):
        dijk, dval, cnt = nv.decompress(m, prec)
        dijk, dval = dijk.cpu().numpy(), dval.cpu().numpy()
        assert cnt == [ref["n"]]
        assert np.array_equal(dijk, ref["ijk"])            # topology + canonical compaction order, exact
        want, scale = oracle_forward_scale(om, 2, dijk)
        if prec == 0:
            assert rel_err(dval / 3.0, want, scale).max() <= FP32_TOL
        else:
            tc_check(prec, om, 2, dijk, dval / 3.0)


def test_patches_match_oracle_decisions(sphere128):
    ijk, val, ref = sphere128
    m = nv.compress(_grid(ijk, val), seed=6, ffm_sigma=1.25, steps=30, batch=2048, patch_precs=1)
    om = blob.read(m.export())
    gp = om["patches"][0]
    l1c = codec.l1_candidates(ref["l1_origin"])
    l0c = codec.l0_candidates(ref["leaf_origin"])
    for net, cand, off, idx, per, truth in (
            (0, l1c, gp["l1_off"], gp["l1_idx"], 4096, vdb.mask_bits(ref["l1_mask"]).reshape(-1)),
            (1, l0c, gp["l0_off"], gp["l0_idx"], 512, vdb.mask_bits(ref["leaf_mask"]).reshape(-1))):
        y, scale = oracle_forward_scale(om, net, cand)
        mism = np.zeros(len(cand), bool)
        rows = np.repeat(np.arange(len(off) - 1), np.diff(off.astype(np.int64)))
        mism[rows * per + idx.astype(np.int64)] = True
        pred_gpu = truth ^ mism
        pred_ref = y > 0
        diff = pred_gpu != pred_ref
        near = np.abs(y) < 4 * FP32_TOL * np.maximum(scale, 1e-30)
        assert not np.any(diff & ~near)                     # only near-zero logits may differ
        assert diff.sum() <= max(2, 1e-4 * len(cand))


def test_import_rejects_corrupt_blobs(sphere128):
    """Blob checks (header on the host; patch offsets and indices on the device): any
    inconsistency is NVDB_ERR_CORRUPT and no model is returned."""
    ijk, val, ref = sphere128
    m = nv.compress(_grid(ijk, val), steps=5, batch=512, patch_precs=0b1001)
    good = m.export()
    assert nv.model_import(good).export() == good               # round trip, bit for bit
    om = blob.read(good)
    cases = []
    bad = blob.read(good)
    bad["patches"][0]["l0_idx"] = bad["patches"][0]["l0_idx"].copy()
    bad["patches"][0]["l0_idx"][0] = 600                      # index >= 512 candidates of a leaf
    cases.append(blob.write(bad))
    bad = blob.read(good)
    off = bad["patches"][3]["l1_off"].copy()
    if len(off) > 2 and off[-1] > 0:
        off[1] = off[-1] + 1                                  # not monotone (and past the list)
        bad["patches"][3]["l1_off"] = off
        cases.append(blob.write(bad))
    bad = blob.read(good)
    off = bad["patches"][0]["l0_off"].copy()
    off[0] = 1                                                # does not start at 0
    bad["patches"][0]["l0_off"] = off
    cases.append(blob.write(bad))
    cases.append(good[:len(good) // 2])                       # truncated
    cases.append(b"NVDBMDL0" + good[8:])                      # wrong magic
    for c in cases:
        with pytest.raises(nv.NvdbError) as e:
            nv.model_import(c)
        assert e.value.status == 8
    assert sorted(om["patches"]) == [0, 3]


def test_decompress_errors(sphere128):
    ijk, val, ref = sphere128
    m = nv.compress(_grid(ijk, val), steps=5, batch=512, patch_precs=1)
    small = (torch.empty((10, 3), dtype=torch.int32, device="cuda"), torch.empty(10, device="cuda"))
    with pytest.raises(nv.NvdbError) as e:
        nv.decompress(m, 0, out=small)
    assert e.value.status == 4
    with pytest.raises(nv.NvdbError) as e:
        nv.decompress(m, 1)                               # no BF16 patch set
    assert e.value.status == 7
    with pytest.raises(nv.NvdbError) as e:
        nv.decompress(m, 2)                               # no FP8 patch set
    assert e.value.status == 7
    with pytest.raises(nv.NvdbError) as e:
        nv.decompress(m, 5)                               # no such precision
    assert e.value.status == 7
    with pytest.raises(nv.NvdbError) as e:
        nv.compress(_grid(ijk, val), steps=1, batch=512, patch_precs=1 << 5)
    assert e.value.status == 1


# ---------------------------------------------------------------------------- query

@pytest.mark.parametrize("prec", [0, 1, 3, 4])
def test_query_parity(sphere128, prec):
    ijk, val, ref = sphere128
    m = nv.compress(_grid(ijk, val), seed=8, ffm_sigma=1.25, steps=100, batch=4096)
    om = blob.read(m.export())
    pts = query_points(torch.from_numpy(ijk), 20000, seed=11).numpy()
    pts = np.concatenate([pts, ref["ijk"][:500].astype(np.float32), np.array([[0.5, 0.5, 0.5]], np.float32)])
    out, act = nv.query(m, _cuda(pts, torch.float32), prec, active=True)
    out, act = out.cpu().numpy(), act.cpu().numpy()
    keys = np.sort(vdb.canonical_key(ref["ijk"]))
    want, bits = codec.query(om, pts, keys)
    assert np.array_equal(act, bits)
    tol = FP32_TOL if prec == 0 else tc_bar(prec)
    assert (np.abs(out - want) / np.maximum(np.abs(want), 3.0)).max() <= tol
    assert (bits != 0).sum() > 1000 and (bits == 0).sum() > 1000


# ---------------------------------------------------------------------------- the learned part

def test_trained_networks_gain_over_untrained(sphere128):
    """Training on the GPU makes the classifiers replace most explicit mask bits and the regressor the values."""
    ijk, val, ref = sphere128
    g = _grid(ijk, val)
    untrained = nv.compress(g, seed=2, ffm_sigma=1.25, steps=0, patch_precs=1)
    trained = nv.compress(g, seed=2, ffm_sigma=1.25, steps=200, batch=4096, patch_precs=1)
    pu, pt = blob.read(untrained.export())["patches"][0], blob.read(trained.export())["patches"][0]
    n_u = int(pu["l0_off"][-1]) + int(pu["l1_off"][-1])
    n_t = int(pt["l0_off"][-1]) + int(pt["l1_off"][-1])
    assert n_t < 0.5 * n_u
    _, dval, _ = nv.decompress(trained, 0)
    dval = dval.cpu().numpy()
    rmse = codec.rmse(ref["val"], dval)
    assert rmse < 0.5 * float(np.std(ref["val"]))       # beats the best constant predictor by 2x
    assert codec.iou_sdf(ref["val"], dval) > 0.85
