"""Pins of oracle/moe.py, the sparse domain decomposition of Section 3.4 (CPU only).

Fixed by the definition rather than by retyping it: constant experts reproduce their
constant (blended values of equal constants) and a weighted average otherwise; a point
deep inside a subdomain sees only its own expert; the gates of two neighbours are mirror
images across their shared face and sum to one over the overlap; the support of an expert
ends exactly halo voxels past its subdomain; at most eight experts share a point; and a
decomposition whose grid has one subdomain reproduces the undecomposed network.
"""
import numpy as np
import pytest

from oracle import codec, moe, vdb
from oracle import nets as N


def _two_blobs():
    """Two small spheres, one on each side of the x = 512 subdomain face of a 1024 domain,
    one of them straddling the face (so the halo region has voxels)."""
    pts = []
    for c, r in (((508.0, 300.0, 300.0), 9.0), ((700.0, 700.0, 520.0), 7.0)):
        a = [np.arange(int(v - r - 4), int(v + r + 4)) for v in c]
        g = np.stack(np.meshgrid(*a, indexing="ij"), -1).reshape(-1, 3)
        d = np.sqrt(((g - np.array(c)) ** 2).sum(1)) - r
        sel = np.abs(d) < 3.0
        pts.append((g[sel], d[sel]))
    # two corner voxels pin the domain to [0, 1024)^3 (origin 0, extent 1024)
    ijk = np.concatenate([p[0] for p in pts] + [np.array([[0, 0, 0], [1023, 1023, 1023]])]).astype(np.int64)
    val = np.concatenate([p[1] for p in pts] + [np.array([1.0, 1.0])]).astype(np.float32)
    return vdb.build(ijk, val)


@pytest.fixture(scope="module")
def grid():
    return _two_blobs()


def _model(grid, **kw):
    opts = codec.default_opts(width=[8, 8, 8], layers=[2, 2, 2], sigma=1.0, subdomain=512, halo=8, **kw)
    return codec.init_model(grid, 0, 3.0, opts)


def test_plan_keeps_occupied_subdomains(grid):
    m = _model(grid)
    p = m["moe"]
    assert p["dims"] == (2, 2, 2)              # the domain extent is 1024
    occupied = {tuple(((c - m["origin"]) // 512).tolist()) for c in grid["ijk"]}
    kept = {tuple(((o - m["origin"]) // 512).tolist()) for o in p["origins"]}
    assert kept == occupied and len(m["nets"]) == 3 * len(kept)
    # origins in lexicographic order of the grid index, expert ids matching
    assert [tuple(o) for o in p["origins"]] == sorted(tuple(o) for o in p["origins"])


def test_gate_values():
    S, h, a = 512, 8, 512
    c = np.array([a - 9, a - 8, a - 1, a, a + 7, a + 8, a + 300, a + S - 9, a + S - 8, a + S + 7, a + S + 8])
    g = moe.gate_axis(c, a, S, h)
    assert np.array_equal(g, [0.0, 0.5 / 16, 7.5 / 16, 8.5 / 16, 15.5 / 16, 1.0, 1.0, 1.0, 15.5 / 16, 0.5 / 16, 0.0])
    # neighbours: the one ending at a and the one starting at a sum to one, mirror images
    x = np.arange(a - 20, a + 20)
    left, right = moe.gate_axis(x, a - S, S, h), moe.gate_axis(x, a, S, h)
    assert np.array_equal(left + right, np.ones_like(left))
    assert np.array_equal(right[20:], left[:20][::-1])


def test_point_deep_inside_sees_only_its_expert(grid):
    m = _model(grid)
    deep = grid["ijk"][np.all((grid["ijk"] % 512 >= 20) & (grid["ijk"] % 512 < 490), axis=1)][:50]
    ids, gs = moe.experts_at(m, codec.REG, deep)
    assert np.all(ids[:, 1:] == -1) and np.all(gs[:, 0] == 1.0)
    own = (deep - m["origin"]) // 512
    flat = (own[:, 0] * 2 + own[:, 1]) * 2 + own[:, 2]
    assert np.array_equal(ids[:, 0], m["moe"]["expert_of"][flat])


def test_constant_experts_blend_to_their_average(grid):
    m = _model(grid)
    n_exp = len(m["moe"]["origins"])
    consts = 0.25 + np.arange(n_exp)
    for k in range(n_exp):
        for j in range(3):
            net = m["nets"][3 * k + j]
            net["W"] = [np.zeros_like(W) for W in net["W"]]
            net["wh"] = np.zeros_like(net["wh"])
            net["bh"] = float(consts[k])
    # straddling points: the gate-weighted average of the experts' constants
    near = grid["ijk"][np.abs(grid["ijk"][:, 0] - 512) < 8]
    assert len(near) > 10
    y = codec.evaluate(m, codec.REG, near)
    ids, gs = moe.experts_at(m, codec.REG, near)
    want = (np.where(ids >= 0, consts[np.maximum(ids, 0)], 0) * gs).sum(1) / gs.sum(1)
    assert np.allclose(y, want, rtol=0, atol=1e-15)
    assert np.all((ids >= 0).sum(1) >= 2)            # both sides of the face contribute
    # equal constants: exactly that constant everywhere
    for k in range(n_exp):
        m["nets"][3 * k + 2]["bh"] = 0.75
    assert np.all(codec.evaluate(m, codec.REG, grid["ijk"]) == 0.75)


def test_at_most_eight_experts_and_support_edges():
    # a voxel set filling the 8 subdomains around the corner (512, 512, 512) of a 1024 domain
    a = np.arange(500, 524)
    g = np.stack(np.meshgrid(a, a, a, indexing="ij"), -1).reshape(-1, 3)
    grid = vdb.build(np.concatenate([g, [[0, 0, 0], [1023, 1023, 1023]]]), np.zeros(len(g) + 2, np.float32))
    m = _model(grid)
    ids, gs = moe.experts_at(m, codec.REG, np.array([[511, 511, 511], [504, 504, 504], [503, 510, 510]]))
    assert (ids[0] >= 0).sum() == 8 and gs[0].sum() == pytest.approx(1.0, abs=0)
    assert (ids[1] >= 0).sum() == 8
    assert (ids[2] >= 0).sum() == 4                    # x = 503 is outside the halo of the x >= 512 side
    lo, hi = moe.support_box(m, int(m["moe"]["expert_of"][0]), codec.REG)
    assert list(lo) == [-8, -8, -8] and list(hi) == [520, 520, 520]
    lo1, hi1 = moe.support_box(m, int(m["moe"]["expert_of"][0]), codec.L1CLS)
    assert list(lo1) == [-1, -1, -1] and list(hi1) == [65, 65, 65]


def test_single_subdomain_equals_undecomposed():
    """A grid whose voxels lie in one subdomain: one expert, gate 1 everywhere it is used,
    the undecomposed forward pass on coordinates relative to the subdomain origin."""
    a = np.arange(100, 130)
    g = np.stack(np.meshgrid(a, a, a, indexing="ij"), -1).reshape(-1, 3)
    d = np.sqrt(((g - 115.0) ** 2).sum(1)) - 10.0
    sel = np.abs(d) < 3
    grid = vdb.build(g[sel], d[sel].astype(np.float32))
    m = _model(grid)
    assert len(m["moe"]["origins"]) == 1
    y = codec.evaluate(m, codec.REG, grid["ijk"])
    z = N.encode(grid["ijk"] - m["moe"]["origins"][0][None], m["q"][1])
    want, _ = N.forward(m["nets"][2], z)
    assert np.allclose(y, want, rtol=0, atol=1e-14)


def test_expert_populations_cover_their_support(grid):
    m = _model(grid)
    for k in range(len(m["moe"]["origins"])):
        lo, hi = moe.support_box(m, k, codec.REG)
        pop = moe.population(grid, m, k, codec.REG)
        inside = np.all((grid["ijk"] >= lo) & (grid["ijk"] < hi), axis=1)
        assert np.array_equal(np.sort(pop), np.nonzero(inside)[0])
        leaves = np.unique(moe.population(grid, m, k, codec.L0CLS) // 512)
        lo_ = grid["leaf_origin"]
        assert np.array_equal(leaves, np.nonzero(np.all((lo_ >= lo) & (lo_ + 8 <= hi), axis=1))[0])
        cand = moe.population(grid, m, k, codec.L1CLS)
        ijk, _ = codec.population(grid, m, codec.L1CLS, cand)
        lo1, hi1 = moe.support_box(m, k, codec.L1CLS)
        assert np.all(((ijk >> 3) >= lo1) & ((ijk >> 3) < hi1))


def test_decomposed_codec_restores_topology(grid):
    m = _model(grid, steps=3, batch=64)
    for k in range(len(m["moe"]["origins"])):
        for net in range(3):
            codec.train_net(grid, m, net, dict(m.get("opts", {}), **codec.default_opts(steps=3, batch=64, sigma=1.0)), expert=k)
    codec.make_patches(grid, m)
    l1o, leafo, act, _ = codec.decode_topology(m)
    assert np.array_equal(leafo, grid["leaf_origin"]) and np.array_equal(act, vdb.mask_bits(grid["leaf_mask"]))
    ijk, val = codec.decompress(m)
    assert np.array_equal(ijk, grid["ijk"])


def test_blob_roundtrip_with_experts(grid):
    from oracle import blob
    m = _model(grid)
    codec.make_patches(grid, m)
    b = blob.write(m)
    r = blob.read(b)
    assert r["moe"]["size"] == 512 and r["moe"]["halo"] == 8 and r["moe"]["dims"] == (2, 2, 2)
    assert np.array_equal(r["moe"]["expert_of"], m["moe"]["expert_of"])
    assert np.array_equal(r["moe"]["origins"], m["moe"]["origins"])
    assert len(r["nets"]) == len(m["nets"])
    for a, c in zip(m["nets"], r["nets"]):
        assert np.array_equal(N.flatten(a).astype(np.float32), N.flatten(c))
    pts = grid["ijk"][::7]
    assert np.allclose(codec.evaluate(r, 2, pts), codec.evaluate(m, 2, pts), rtol=1e-5, atol=1e-6)
