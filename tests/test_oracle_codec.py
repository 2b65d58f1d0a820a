"""Pins of the oracle's codec: patches, top-down decode, query, blob (CPU only)."""
import numpy as np
import pytest

from fixtures import workload
from oracle import blob, codec, vdb
from oracle import nets as N


def _corner_sphere():
    """Small spherical band straddling 8 level-2 (and level-1) nodes at (4096,4096,4096)."""
    a = np.arange(4084, 4109)
    g = np.stack(np.meshgrid(a, a, a, indexing="ij"), -1).reshape(-1, 3)
    d = np.sqrt(((g - 4096.5) ** 2).sum(1)) - 7.0
    sel = np.abs(d) < 3.0
    return g[sel], d[sel].astype(np.float32)


@pytest.fixture(scope="module", params=["sphere32", "union128", "corner"])
def grid(request):
    if request.param == "corner":
        ijk, val = _corner_sphere()
    else:
        ijk, val, _ = workload(request.param)
        ijk, val = ijk.numpy(), val.numpy()
    return vdb.build(ijk, val)


def _const_net(model, k, bias):
    net = model["nets"][k]
    net["W"] = [np.zeros_like(W) for W in net["W"]]
    net["wh"] = np.zeros_like(net["wh"])
    net["bh"] = bias


def test_decode_restores_topology_for_any_weights(grid):
    opts = codec.default_opts(width=[8, 16, 8], layers=[2, 3, 2], sigma=1.0)
    m = codec.init_model(grid, 0, 3.0, opts)
    codec.make_patches(grid, m)
    l1o, leafo, act, _ = codec.decode_topology(m)
    assert np.array_equal(l1o, grid["l1_origin"])
    assert np.array_equal(leafo, grid["leaf_origin"])
    assert np.array_equal(act, vdb.mask_bits(grid["leaf_mask"]))
    ijk, val = codec.decompress(m)
    assert np.array_equal(ijk, grid["ijk"])


def test_patch_counts_closed_form(grid):
    m = codec.init_model(grid, 0, 3.0, codec.default_opts(width=[8, 8, 8], layers=[1, 1, 1]))
    n_l1, n_leaf, n = grid["l1_origin"].shape[0], grid["leaf_origin"].shape[0], grid["n"]
    _const_net(m, 0, +1.0); _const_net(m, 1, +1.0)       # everything predicted active
    p = codec.make_patches(grid, m)
    assert p["l1_off"][-1] == 4096 * n_l1 - n_leaf and p["l0_off"][-1] == 512 * n_leaf - n
    _const_net(m, 0, -1.0); _const_net(m, 1, -1.0)       # everything predicted inactive
    p = codec.make_patches(grid, m)
    assert p["l1_off"][-1] == n_leaf and p["l0_off"][-1] == n
    assert np.all(np.diff(p["l1_off"].astype(np.int64)) >= 0)
    _const_net(m, 0, 0.0)                                  # logit 0 is inactive (strict threshold)
    assert codec.make_patches(grid, m)["l1_off"][-1] == n_leaf


def test_decoded_values_constant_regressor(grid):
    m = codec.init_model(grid, 0, 3.0, codec.default_opts(width=[8, 8, 8], layers=[1, 1, 1]))
    codec.make_patches(grid, m)
    _const_net(m, 2, 0.25)
    ijk, val = codec.decompress(m)
    assert np.all(val == 0.75)


def test_query_pins(grid):
    m = codec.init_model(grid, 0, 3.0, codec.default_opts(width=[8, 8, 8], layers=[1, 1, 2], sigma=1.0))
    keys = np.sort(vdb.canonical_key(grid["ijk"]))
    # integer points of active voxels reproduce the regressed voxel value
    vox = grid["ijk"][:: max(1, grid["n"] // 200)]
    got, bits = codec.query(m, vox.astype(np.float32), keys)
    want = codec.evaluate(m, codec.REG, vox) * 3.0
    assert np.allclose(got, want, rtol=0, atol=1e-12) and np.all(bits & 1)
    # far from the band: all corners inactive -> background
    far = grid["ijk"].min(0) - 40
    far = np.maximum(far, 0).astype(np.float32)[None] + np.array([[0.3, 0.6, 0.9]], np.float32)
    got, bits = codec.query(m, far, keys)
    if bits[0] == 0:
        assert got[0] == pytest.approx(3.0, abs=1e-12)
    # cell centre with all 8 corners active: mean of the corner values
    s = set(map(tuple, grid["ijk"].tolist()))
    cells = [p for p in grid["ijk"][:5000] if all((p[0] + a, p[1] + b, p[2] + c) in s
                                                     for a in (0, 1) for b in (0, 1) for c in (0, 1))][:20]
    assert cells, "no fully active cell"
    cells = np.array(cells)
    got, bits = codec.query(m, (cells + 0.5).astype(np.float32), keys)
    assert np.all(bits == 255)
    corners = np.array([[a, b, c] for a in (0, 1) for b in (0, 1) for c in (0, 1)])
    vals = np.stack([codec.evaluate(m, codec.REG, cells + o) * 3.0 for o in corners], 1)
    assert np.allclose(got, vals.mean(1), rtol=0, atol=1e-12)
    # linear along an x edge when both ends are active (other corners weigh 0)
    t = np.array([0.25], np.float32)
    p = cells[:1].astype(np.float32) + np.stack([t, 0 * t, 0 * t], 1)
    got, _ = codec.query(m, p, keys)
    assert got[0] == pytest.approx(0.75 * vals[0, 0] + 0.25 * vals[0, 4], abs=1e-12)


def test_constant_regressor_query_is_exact():
    ijk, val, _ = workload("sphere32")
    g = vdb.build(ijk.numpy(), val.numpy())
    m = codec.init_model(g, 0, 3.0, codec.default_opts(width=[8, 8, 8], layers=[1, 1, 1]))
    _const_net(m, 2, -0.5)
    keys = np.sort(vdb.canonical_key(g["ijk"]))
    pts = g["ijk"][::37].astype(np.float32) + np.float32(0.37)
    got, bits = codec.query(m, pts, keys)
    # trilinear weights sum to one: result = sum over corners of (-1.5 if active else +3)
    wsum = np.zeros(len(pts))
    t = pts.astype(np.float64) - np.floor(pts)
    for c in range(8):
        w = np.ones(len(pts))
        for d, b in enumerate(((c >> 2) & 1, (c >> 1) & 1, c & 1)):
            w = w * (t[:, d] if b else 1 - t[:, d])
        wsum += w * np.where((bits >> c) & 1, -1.5, 3.0)
    assert np.allclose(got, wsum, rtol=0, atol=1e-12)


def test_blob_roundtrip(grid):
    m = codec.init_model(grid, 1, 0.0, codec.default_opts(width=[8, 16, 24], layers=[1, 2, 3]))
    codec.make_patches(grid, m, codec.PREC_FP32)
    codec.make_patches(grid, m, codec.PREC_BF16)
    b = blob.write(m)
    assert len(b) % 8 == 0
    r = blob.read(b)
    for k in range(3):
        a, c = N.flatten(m["nets"][k]), N.flatten(r["nets"][k])
        assert np.array_equal(a.astype(np.float32), c)
    assert np.array_equal(r["l2_mask"], grid["l2_mask"]) and np.array_equal(r["q"][1], m["q"][1])
    for prec in (0, 1):
        for key in ("l1_off", "l1_idx", "l0_off", "l0_idx"):
            assert np.array_equal(r["patches"][prec][key], m["patches"][prec][key])


def test_training_reduces_loss():
    ijk, val, _ = workload("sphere32")
    g = vdb.build(ijk.numpy(), val.numpy())
    opts = codec.default_opts(sigma=1.0, steps=60, batch=512, lr=5e-3)
    m = codec.init_model(g, 0, 3.0, opts)
    for k in range(3):
        ls = codec.train_net(g, m, k, opts)
        assert np.mean(ls[-10:]) < 0.8 * np.mean(ls[:10])
