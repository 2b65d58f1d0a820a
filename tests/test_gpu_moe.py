"""Sparse domain decomposition (Section 3.4) on the GPU against the FP64 oracle.

A level set straddling the x = 512 face of a 1024^3 domain (two corner voxels pin the
domain), decomposed into 512^3 subdomains with an 8-voxel halo: the expert table and the
initial experts bit-exact; the gated networks (Eq. 3) at 1e-5 (FP32) and 2e-2 (tensor
cores) of the head scale; the first Adam step of every expert's networks on its support's
samples; topology restored exactly and values at the same bars through decompress and
query; blob round trip.
"""
import numpy as np
import pytest
import torch

import paper_2208_04448_b300 as nv
from gpu_helpers import tc_bar
from oracle import blob, codec, moe, vdb
from oracle import nets as N

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
SEED, SIGMA = 41, 1.25
SHAPE = dict(width=[32, 64, 64], layers=[2, 3, 3])


def _voxels():
    pts = []
    for c, r in (((506.0, 300.0, 300.0), 17.0), ((700.0, 690.0, 515.0), 11.0), ((300.0, 508.0, 700.0), 9.0)):
        a = [np.arange(int(v - r - 4), int(v + r + 4)) for v in c]
        g = np.stack(np.meshgrid(*a, indexing="ij"), -1).reshape(-1, 3)
        d = np.sqrt(((g - np.array(c)) ** 2).sum(1)) - r
        sel = np.abs(d) < 3.0
        pts.append((g[sel], d[sel]))
    ijk = np.concatenate([p[0] for p in pts] + [np.array([[0, 0, 0], [1023, 1023, 1023]])]).astype(np.int32)
    val = np.concatenate([p[1] for p in pts] + [np.array([1.0, 1.0])]).astype(np.float32)
    return ijk, val


@pytest.fixture(scope="module")
def case():
    ijk, val = _voxels()
    ref = vdb.build(ijk, val)
    g = nv.build(torch.from_numpy(ijk).cuda(), torch.from_numpy(val).cuda(), 0, 3.0)
    return ijk, val, ref, g


def _opts(**kw):
    return codec.default_opts(seed=SEED, sigma=SIGMA, subdomain=512, halo=8, **SHAPE, **kw)


def test_expert_table_and_initial_experts(case):
    ijk, val, ref, g = case
    m = nv.compress(g, seed=SEED, ffm_sigma=SIGMA, steps=0, subdomain=512, halo=8, patch_precs=1, **SHAPE)
    info = m.info()
    om = codec.init_model(ref, 0, 3.0, _opts())
    assert info["subdomain"] == 512 and info["n_experts"] == len(om["moe"]["origins"]) >= 4
    got = blob.read(m.export())
    assert got["moe"]["dims"] == om["moe"]["dims"]
    assert np.array_equal(got["moe"]["expert_of"], om["moe"]["expert_of"])
    assert np.array_equal(got["moe"]["origins"], om["moe"]["origins"])
    assert np.array_equal(got["q"][0], om["q"][0]) and np.array_equal(got["q"][1], om["q"][1])
    assert len(got["nets"]) == len(om["nets"])
    for a, b in zip(got["nets"], om["nets"]):
        assert np.array_equal(N.flatten(a), N.flatten(b).astype(np.float32).astype(np.float64))


@pytest.fixture(scope="module")
def trained(case):
    ijk, val, ref, g = case
    m = nv.compress(g, seed=SEED, ffm_sigma=SIGMA, steps=40, batch=2048, subdomain=512, halo=8,
                    patch_precs=0b11011, **SHAPE)
    return m, blob.read(m.export())


def _points(ref):
    r = np.random.default_rng(1)
    near = ref["ijk"][np.abs(ref["ijk"][:, 0] - 512) < 12]           # rows in the halo of the x face
    return np.concatenate([near, ref["ijk"][r.integers(0, ref["n"], 1500)]]).astype(np.int32)


def _blended(om, net, pts):
    """Oracle output (Eq. 3) and its error scale: the gate-weighted head dot-product scales
    sum_i |w_h,i h_i| + |b_h| of the experts."""
    want = codec.evaluate(om, net, pts)
    scale = np.zeros(len(pts))
    ids, gs = moe.experts_at(om, net, pts)
    for k in np.unique(ids[ids >= 0]):
        rows, slots = np.nonzero(ids == k)
        kk = 3 * int(k) + net
        z = N.encode(moe.expert_coords(om, int(k), net, pts[rows]), codec.level_q(om, net))
        _, (hs, _) = N.forward(om["nets"][kk], z)
        s_k = np.abs(hs[-1] * om["nets"][kk]["wh"][None]).sum(1) + abs(om["nets"][kk]["bh"])
        scale[rows] += gs[rows, slots] * s_k
    return want, scale / np.maximum(gs.sum(1), 1e-30)


def _check(prec, got, want, scale):
    if prec == 0:
        err = np.abs(got - want) / np.maximum(np.abs(want), np.maximum(scale, 1e-30))
        assert err.max() <= FP32_TOL, err.max()
    else:
        err = np.abs(got - want) / np.maximum(scale, 1.0)
        assert err.max() <= tc_bar(prec), err.max()


@pytest.mark.parametrize("prec", [0, 1, 3, 4])
def test_gated_networks_match_oracle(case, trained, prec):
    ijk, val, ref, g = case
    m, om = trained
    pts = _points(ref)
    ids, _ = moe.experts_at(om, 2, pts)
    assert ((ids >= 0).sum(1) >= 2).sum() > 100                       # many rows blend two experts
    for net in range(3):
        want, scale = _blended(om, net, pts)
        got = nv.mlp_eval(m, net, torch.from_numpy(pts).cuda(), prec).cpu().numpy()
        _check(prec, got, want, scale)


def test_first_adam_step_of_every_expert(case):
    ijk, val, ref, g = case
    m = nv.compress(g, seed=SEED, ffm_sigma=SIGMA, steps=1, batch=2048, lr=1e-3, subdomain=512, halo=8,
                    patch_precs=1, **SHAPE)
    opts = _opts(steps=1, batch=2048, lr=1e-3)
    om = codec.init_model(ref, 0, 3.0, opts)
    theta0 = [N.flatten(n) for n in om["nets"]]
    got = blob.read(m.export())
    for e in range(len(om["moe"]["origins"])):
        for net in range(3):
            kk = 3 * e + net
            ls = codec.train_net(ref, om, net, opts, expert=e)
            assert abs(m.losses(kk)[0] - ls[0]) <= 1e-5 * max(1.0, abs(ls[0])), (e, net)   # same samples
            dw_ref = N.flatten(om["nets"][kk]) - theta0[kk]
            dw_got = N.flatten(got["nets"][kk]) - theta0[kk]
            # components whose FP64 gradient is resolved in FP32 (|g| > ~1e-5, i.e. the first
            # step within 0.1% of lr): the steps agree; smaller ones may change sign
            big = np.abs(dw_ref) > 0.999e-3
            assert big.sum() > 0
            assert np.abs(dw_got[big] - dw_ref[big]).max() <= 2e-6, (e, net)


@pytest.mark.parametrize("prec", [0, 3, 1])
def test_decompress_and_query(case, trained, prec):
    ijk, val, ref, g = case
    m, om = trained
    dijk, dval, cnt = nv.decompress(m, prec)
    dijk, dval = dijk.cpu().numpy(), dval.cpu().numpy()
    assert cnt == [ref["n"]] and np.array_equal(dijk, ref["ijk"])     # topology exact, canonical order
    want, scale = _blended(om, 2, dijk)
    _check(prec, dval / 3.0, want, scale)
    if prec == 0:
        r = np.random.default_rng(4)
        pts = (ref["ijk"][r.integers(0, ref["n"], 3000)] + r.random((3000, 3))).astype(np.float32)
        out, act = nv.query(m, torch.from_numpy(pts).cuda(), prec, active=True)
        wq, bits = codec.query(om, pts, np.sort(vdb.canonical_key(ref["ijk"])))
        assert np.array_equal(act.cpu().numpy(), bits)
        assert np.abs(out.cpu().numpy() - wq).max() <= 1e-4


def test_blob_roundtrip_decodes_identically(case, trained):
    ijk, val, ref, g = case
    m, om = trained
    m2 = nv.model_import(m.export())
    a = nv.decompress(m, 3)
    b = nv.decompress(m2, 3)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    bad = bytearray(m.export())
    bad[112:120] = (500).to_bytes(8, "little")    # subdomain size not a multiple of 512
    with pytest.raises(nv.NvdbError) as e:
        nv.model_import(bytes(bad))
    assert e.value.status == nv.ERR_CORRUPT
