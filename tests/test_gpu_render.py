"""Ray marching on the GPU (nvdb_render, Section 4's ray-marched cloud) against the FP64
oracle renderer on the same model: radiance and transmittance per pixel."""
import numpy as np
import pytest
import torch

import paper_2208_04448_b300 as nv
from fixtures import workload
from oracle import blob, render, vdb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fog():
    ijk, val, _ = workload("fog64")
    ref = vdb.build(ijk.numpy(), val.numpy())
    g = nv.build(ijk.cuda().contiguous(), val.cuda().contiguous(), 1, 0.0)
    m = nv.compress(g, seed=9, ffm_sigma=1.25, steps=150, batch=8192, patch_precs=0b11001)
    return ref, m, blob.read(m.export())


CAM = dict(eye=[140.0, 90.0, -60.0], target=[32.0, 32.0, 32.0], up=[0.0, 1.0, 0.0], fov_deg=35.0,
           width=24, height=20, step=1.7, max_steps=160, sigma=0.08)


@pytest.mark.parametrize("prec", [nv.FP32, nv.FP16])
def test_render_matches_oracle(fog, prec):
    ref, m, om = fog
    img = nv.render(m, prec=prec, **CAM).cpu().numpy().astype(np.float64)
    want = render.render(om, CAM, np.sort(vdb.canonical_key(ref["ijk"])))
    assert want[..., 0].max() > 0.05 and want[..., 1].min() < 0.9      # the cloud is in view
    assert (want[..., 1] == 1.0).any()                                   # and some rays miss it
    tol = 2e-4 if prec == nv.FP32 else 2e-2
    assert np.abs(img[..., 0] - want[..., 0]).max() <= tol * want[..., 0].max()
    assert np.abs(img[..., 1] - want[..., 1]).max() <= tol
