"""Batched decode (many models per stage launch) and graph-captured decode plans."""
import numpy as np
import pytest
import torch

import paper_2208_04448_b300 as nv
from fixtures import workload

pytestmark = pytest.mark.gpu


def _grid(name):
    if name == "corner":
        a = np.arange(4084, 4109)
        g = np.stack(np.meshgrid(a, a, a, indexing="ij"), -1).reshape(-1, 3)
        d = np.sqrt(((g - 4096.5) ** 2).sum(1)) - 7.0
        sel = np.abs(d) < 3.0
        ijk, val = torch.from_numpy(g[sel].astype(np.int32)), torch.from_numpy(d[sel].astype(np.float32))
    else:
        ijk, val, _ = workload(name)
    return nv.build(ijk.cuda().contiguous(), val.cuda().contiguous(), 0, 3.0)


@pytest.fixture(scope="module")
def models():
    shape = dict(width=[32, 64, 64], layers=[3, 3, 4], ffm_size=[32, 64], ffm_sigma=1.25, batch=2048)
    ms = [nv.compress(_grid(n), seed=i + 1, steps=20, **shape) for i, n in enumerate(["sphere32", "union128", "corner"])]
    other = nv.compress(_grid("sphere32"), seed=9, steps=5, batch=1024)   # default 3x32 shapes
    return ms, other


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_batched_equals_single(models, prec):
    ms, other = models
    singles = [nv.decompress(m, prec) for m in ms + [other]]
    ijk, val, counts = nv.decompress(ms + [other, ms[0]], prec)     # 3 same-shape runs + other shape + repeat
    assert counts == [s[2][0] for s in singles] + [singles[0][2][0]]
    off = 0
    for s in singles + [singles[0]]:
        n = s[2][0]
        assert torch.equal(ijk[off:off + n], s[0]) and torch.equal(val[off:off + n], s[1])
        off += n


@pytest.mark.parametrize("pinned", [True, False])
def test_decompress_to_host_equals_device_decode(models, pinned):
    ms, other = models
    seq = ms + [other, ms[0]]                                        # several runs: one host copy per run
    ijk, val, counts = nv.decompress(seq, 3)
    total = sum(counts)
    host = (torch.full((total + 5, 3), -1, dtype=torch.int32, pin_memory=pinned),
            torch.full((total + 5,), -1.0, dtype=torch.float32, pin_memory=pinned))
    hijk, hval, hcounts = nv.decompress_host(seq, 3, host=host)
    assert hcounts == counts
    assert torch.equal(hijk, ijk.cpu()) and torch.equal(hval, val.cpu())
    assert (host[0][total:] == -1).all() and (host[1][total:] == -1.0).all()   # nothing past the result
    single = nv.decompress_host(ms[1], 1)                           # allocates pinned host buffers itself
    ref = nv.decompress(ms[1], 1)
    assert torch.equal(single[0], ref[0].cpu()) and torch.equal(single[1], ref[1].cpu())
    with pytest.raises(ValueError):
        nv.decompress_host(seq, 3, host=(host[0][:10], host[1]))


def test_more_models_than_one_launch_holds(models):
    ms, _ = models
    seq = [ms[i % 3] for i in range(50)]                              # > 48: two launches per stage
    ijk, val, counts = nv.decompress(seq, 3)
    ref = [nv.decompress(m, 3) for m in ms]
    off = 0
    for i, n in enumerate(counts):
        r = ref[i % 3]
        assert torch.equal(ijk[off:off + n], r[0]) and torch.equal(val[off:off + n], r[1])
        off += n


@pytest.mark.parametrize("prec", [1, 3, 4])
def test_plan_replays_decompress(models, prec):
    ms, other = models
    seq = ms + [other]
    plan = nv.decompress_plan(seq, prec)
    info = plan.info()
    assert 0 <= info["tc_ctas_per_sm"] <= 4 and info["tuned_ms"] > 0
    ijk, val, _ = nv.decompress(seq, prec)
    for _ in range(2):
        plan.ijk.zero_(); plan.val.zero_()
        plan.launch()
        plan.check()
        assert torch.equal(plan.ijk, ijk) and torch.equal(plan.val, val)
