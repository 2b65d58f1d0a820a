"""Network shapes at the edges of what the kernels take: one hidden layer, width 32 with a
64-wide encoding, and the deepest tensor-core training step (4 layers), across every
decode precision and both training precisions, against the FP64 oracle."""
import numpy as np
import pytest
import torch

import paper_2208_04448_b300 as nv
from fixtures import workload
from gpu_helpers import oracle_forward_scale, rel_err, tc_check
from oracle import blob, codec, vdb
from oracle import nets as N

pytestmark = pytest.mark.gpu

SHAPES = [
    dict(width=[32, 32, 32], layers=[1, 1, 1], ffm_size=[32, 32]),
    dict(width=[64, 32, 64], layers=[1, 2, 1], ffm_size=[64, 64]),
    dict(width=[32, 32, 64], layers=[4, 4, 4], ffm_size=[64, 64]),
]


@pytest.fixture(scope="module")
def union():
    ijk, val, _ = workload("union128")
    ijk, val = ijk.numpy(), val.numpy()
    return ijk, val, vdb.build(ijk, val)


@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("train_prec", [0, 1])
def test_shapes_train_and_decode(union, shape, train_prec):
    ijk, val, ref = union
    g = nv.build(torch.from_numpy(ijk).cuda().contiguous(), torch.from_numpy(val).cuda().contiguous(), 0, 3.0)
    m = nv.compress(g, seed=2, ffm_sigma=1.25, steps=60, batch=4096, train_prec=train_prec, **SHAPES[shape])
    for k in range(3):
        ls = m.losses(k)
        assert len(ls) == 60 and np.all(np.isfinite(ls))
    om = blob.read(m.export())
    want, scale = oracle_forward_scale(om, codec.REG, ref["ijk"])
    for prec in (0, 1, 2, 3, 4):
        dijk, dval, cnt = nv.decompress(m, prec)
        assert cnt == [ref["n"]] and np.array_equal(dijk.cpu().numpy(), ref["ijk"])
        if prec == 0:
            assert rel_err(dval.cpu().numpy() / 3.0, want, scale).max() <= 1e-5
        else:
            tc_check(prec, om, codec.REG, ref["ijk"], dval.cpu().numpy() / 3.0)


@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_shapes_gradients(union, shape):
    ijk, val, ref = union
    g = nv.build(torch.from_numpy(ijk).cuda().contiguous(), torch.from_numpy(val).cuda().contiguous(), 0, 3.0)
    m = nv.compress(g, seed=4, ffm_sigma=1.25, steps=0, patch_precs=1, **SHAPES[shape])
    om = blob.read(m.export())
    r = np.random.default_rng(shape)
    pts = ref["ijk"][r.integers(0, ref["n"], 700)].astype(np.int32)
    tgt = r.standard_normal(len(pts)).astype(np.float32)
    for net in range(3):
        y, cache = N.forward(om["nets"][net], N.encode(codec.level_coords(om, net, pts), codec.level_q(om, net)))
        lref, gy = N.loss_and_grad(y, tgt.astype(np.float64), 0)
        gref = N.flatten(N.backward(om["nets"][net], cache, gy))
        g32, _ = nv.mlp_grad(m, net, torch.from_numpy(pts).cuda(), torch.from_numpy(tgt).cuda(), 0, 0)
        assert np.abs(g32.cpu().numpy() - gref).max() <= 1e-4 * np.abs(gref).max()
        g16, _ = nv.mlp_grad(m, net, torch.from_numpy(pts).cuda(), torch.from_numpy(tgt).cuda(), 0, 1)
        assert np.linalg.norm(g16.cpu().numpy() - gref) <= 0.1 * np.linalg.norm(gref)
