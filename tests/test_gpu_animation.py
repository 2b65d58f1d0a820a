"""Animated volumes (Section 3.6): temporally coherent warm start with early stop, and
the batched decode of all frames in one graph-captured plan."""
import numpy as np
import pytest
import torch

import paper_2208_04448_b300 as nv
from fixtures import water_frame
from gpu_helpers import oracle_forward_scale, rel_err, tc_bar
from oracle import blob, codec
from oracle import nets as N

pytestmark = pytest.mark.gpu

SHAPE = dict(width=[32, 64, 64], layers=[3, 3, 3], ffm_size=[32, 64], ffm_sigma=2.0, batch=8192)


@pytest.fixture(scope="module")
def frames():
    out = []
    for f in range(6):
        ijk, val = water_frame(f, nx=256, ny=64, nz=256, y0=32.0, device="cuda")
        out.append((ijk.contiguous(), val.contiguous()))
    return out


def test_warm_start_copies_previous_networks(frames):
    g0 = nv.build(*frames[0], 0, 3.0)
    g1 = nv.build(*frames[1], 0, 3.0)
    m0 = nv.compress(g0, seed=1, steps=40, patch_precs=1, **SHAPE)
    w = nv.compress(g1, seed=99, steps=0, patch_precs=1, warm=m0, **SHAPE)
    a, b = blob.read(m0.export()), blob.read(w.export())
    for k in range(3):
        assert np.array_equal(N.flatten(a["nets"][k]), N.flatten(b["nets"][k]))
    assert np.array_equal(a["q"][0], b["q"][0]) and np.array_equal(a["q"][1], b["q"][1])


def test_warm_sequence_early_stop_and_batched_decode(frames):
    cold = nv.compress(nv.build(*frames[0], 0, 3.0), seed=1, steps=600, lr=1e-3, patch_precs=0b11011, **SHAPE)
    target = [float(np.mean(cold.losses(k)[-50:])) for k in range(3)]
    models, grids_ijk, steps = [cold], [frames[0][0]], []
    for f in range(1, len(frames)):
        g = nv.build(*frames[f], 0, 3.0)
        m = nv.compress(g, seed=1, steps=600, lr=1e-4, warm=models[-1], patch_precs=0b11011, stop_window=50,
                        stop_loss=target, **SHAPE)
        steps.append([len(m.losses(k)) for k in range(3)])
        models.append(m)
        grids_ijk.append(g.read()["ijk"])
    warm_steps = np.array(steps)
    assert warm_steps.max() <= 600 and warm_steps.sum() < 0.8 * 3 * 600 * (len(frames) - 1)
    assert (warm_steps < 600).any()                       # the early stop triggered
    for prec in (1, 3, 4):
        plan = nv.decompress_plan(models, prec)
        plan.launch()
        plan.check()
        ijk, val, counts = nv.decompress(models, prec)
        assert torch.equal(plan.ijk, ijk) and torch.equal(plan.val, val)
        off = 0
        for f, n in enumerate(counts):
            ref = grids_ijk[f] if f else nv.build(*frames[0], 0, 3.0).read()["ijk"]
            assert np.array_equal(ijk[off:off + n].cpu().numpy(), ref)   # every frame's topology, exact
            # and every frame's values, warm-started ones included, against the oracle on the
            # frame's own (warm-trained) weights
            om = blob.read(models[f].export())
            idx = np.random.default_rng(f).choice(n, 2048, replace=False)
            pv = val[off:off + n][torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64) / 3.0
            want, scale = oracle_forward_scale(om, codec.REG, ref[idx])
            assert np.abs(pv - want).max() <= tc_bar(prec), (f, prec)
            off += n
