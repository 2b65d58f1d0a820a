"""Explicit-grid samplers (order 0 / 1 / 3), isosurface points and mCD (Eq. 4) on the GPU
against oracle/sample.py; and mCD of a decoded model against its source."""
import numpy as np
import pytest
import torch

import paper_2208_04448_b300 as nv
from fixtures import workload
from oracle import sample, vdb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["sphere32", "union128"])
def grid(request):
    ijk, val, _ = workload(request.param)
    ref = vdb.build(ijk.numpy(), val.numpy())
    return ref, nv.build(ijk.cuda().contiguous(), val.cuda().contiguous(), 0, 3.0)


@pytest.mark.parametrize("order", [0, 1, 3])
def test_samplers_match_oracle(grid, order):
    ref, g = grid
    r = np.random.default_rng(order)
    p = (ref["ijk"][r.integers(0, ref["n"], 4000)] + r.uniform(-1.5, 1.5, (4000, 3))).astype(np.float32)
    got = nv.grid_sample(g, torch.from_numpy(p).cuda(), order).cpu().numpy()
    want = sample.sample(ref, 3.0, p, order)
    assert np.abs(got - want).max() <= 2e-5


def test_isosurface_and_mcd_match_oracle(grid):
    ref, g = grid
    got = nv.grid_isosurface(g).cpu().numpy()
    want = sample.isosurface(ref, 3.0)
    assert got.shape == want.shape and np.abs(got - want).max() <= 2e-5   # FP32 positions (~1e2 voxels)
    # a reconstruction: the same voxels, values moved by a smooth field
    ijk = ref["ijk"]
    val = ref["val"] + (0.05 * np.sin(ijk[:, 0] / 7.0)).astype(np.float32)
    ref2 = vdb.build(ijk, val)
    g2 = nv.build(torch.from_numpy(ijk.astype(np.int32)).cuda(), torch.from_numpy(val).cuda(), 0, 3.0)
    m = nv.mcd(g, g2)
    assert abs(m - sample.mcd(ref, ref2, 3.0)) <= 1e-5 * max(1.0, m)
    # a grid against itself: the trilinear value at its own FP32 crossing points is zero up to
    # the rounding of (1 - t) v0 + t v1 (a few ulp of |v| <= 3)
    assert nv.mcd(g, g) <= 2e-6


def test_mcd_of_a_decoded_model():
    ijk, val, _ = workload("sphere128")
    g = nv.build(ijk.cuda().contiguous(), val.cuda().contiguous(), 0, 3.0)
    m = nv.compress(g, seed=3, ffm_sigma=1.25, steps=300, batch=4096, patch_precs=1 << nv.FP16)
    dijk, dval, _ = nv.decompress(m, nv.FP16)
    rec = nv.build(dijk.contiguous(), dval.contiguous(), 0, 3.0)
    d = nv.mcd(g, rec)
    print("mCD of the decoded sphere:", d)
    assert 0.0 < d < 0.5
