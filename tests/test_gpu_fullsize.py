"""Parity at the benchmark's full size (1024^3 union of 64 primitives, 4x64 networks),
in the launch configuration bench.py times: the whole decode is checked exactly for
topology and order; values and point queries are checked on sampled outputs that the
FP64 oracle computes one by one."""
import numpy as np
import pytest
import torch

import paper_2208_04448_b300 as nv
from fixtures import workload
from gpu_helpers import oracle_forward_scale, rel_err, tc_check
from oracle import blob, codec, vdb

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def union1024():
    ijk, val, _ = workload("union1024", device="cuda")
    g = nv.build(ijk.contiguous(), val.contiguous(), 0, 3.0)
    info = g.info()
    m = nv.compress(g, seed=1, width=[64, 64, 64], layers=[4, 4, 4], ffm_size=[64, 64],
                    ffm_sigma=10.0 * (1 << info["log2_extent"]) / 1024.0, steps=200, batch=65536,
                    patch_precs=0b11111)
    return g, m, g.read()


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_full_decode_topology_and_sampled_values(union1024, prec):
    g, m, ref = union1024
    om = blob.read(m.export())
    dijk, dval, cnt = nv.decompress(m, prec)
    assert cnt == [ref["ijk"].shape[0]] and cnt[0] > 10_000_000
    assert torch.equal(dijk, torch.from_numpy(ref["ijk"]).cuda())     # every voxel, canonical order
    r = np.random.default_rng(prec)
    idx = r.choice(cnt[0], 4096, replace=False)
    pi = ref["ijk"][idx]
    pv = dval[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    want, scale = oracle_forward_scale(om, codec.REG, pi)
    if prec == 0:
        assert rel_err(pv / 3.0, want, scale).max() <= FP32_TOL
    else:
        tc_check(prec, om, codec.REG, pi, pv / 3.0)
    # decoding twice gives identical bits
    dijk2, dval2, _ = nv.decompress(m, prec)
    assert torch.equal(dval, dval2) and torch.equal(dijk, dijk2)


def test_full_size_queries_sampled(union1024):
    g, m, ref = union1024
    om = blob.read(m.export())
    from fixtures import query_points
    pts = query_points(torch.from_numpy(ref["ijk"]), 1 << 22, seed=5)
    out, act = nv.query(m, pts.cuda().contiguous(), 0, active=True)
    r = np.random.default_rng(3)
    act_np = act.cpu().numpy()
    near = np.nonzero(act_np)[0]
    idx = np.concatenate([r.choice(near, 1500, replace=False), r.choice(len(act_np), 500, replace=False)])
    keys = np.sort(vdb.canonical_key(ref["ijk"]))
    want, bits = codec.query(om, pts.numpy()[idx], keys)
    assert np.array_equal(act_np[idx], bits)
    got = out.cpu().numpy()[idx]
    assert (np.abs(got - want) / np.maximum(np.abs(want), 3.0)).max() <= FP32_TOL
