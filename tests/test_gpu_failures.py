"""Failure handling without a GPU fault: a bounded device wait that runs out, waits forced
to report a timeout after their phase completed (the kernels' real timeout path, nothing
in flight), and a budget that makes device allocations fail.  Afterwards the device and
the models stay usable and give the same bits as before."""
import numpy as np
import pytest
import torch

import paper_2208_04448_b300 as nv
from fixtures import workload

pytestmark = pytest.mark.gpu

TIMEOUT, OOM = 6, 3


@pytest.fixture(scope="module")
def model():
    ijk, val, _ = workload("sphere32")
    g = nv.build(ijk.cuda().contiguous(), val.cuda().contiguous(), 0, 3.0)
    return g, nv.compress(g, seed=1, ffm_sigma=1.0, steps=20, batch=1024)


def test_bounded_wait_runs_out_and_device_stays_usable(model):
    g, m = model
    ref = nv.decompress(m, nv.FP16)
    with pytest.raises(nv.NvdbError) as e:
        nv.debug_wait_selftest(20_000_000)       # 20 ms on a phase nothing completes
    assert e.value.status == TIMEOUT
    again = nv.decompress(m, nv.FP16)
    assert torch.equal(again[0], ref[0]) and torch.equal(again[1], ref[1])


def test_forced_timeouts_take_the_error_path(model):
    g, m = model
    ref = nv.decompress(m, nv.FP16)
    pts = torch.from_numpy(g.read()["ijk"][:300]).cuda()
    tgt = torch.zeros(300, device="cuda")
    nv.debug_inject(nv.INJECT_WAIT_TIMEOUT, 1)
    try:
        for call in (lambda: nv.decompress(m, nv.FP16),
                     lambda: nv.decompress(m, nv.BF16X3),
                     lambda: nv.query(m, pts.float().contiguous(), nv.FP16),
                     lambda: nv.mlp_eval(m, 2, pts, nv.FP16),
                     lambda: nv.mlp_grad(m, 2, pts, tgt, 0, nv.BF16),
                     lambda: nv.compress(g, steps=3, batch=1024, train_prec=nv.BF16, patch_precs=1)):
            with pytest.raises(nv.NvdbError) as e:
                call()
            assert e.value.status == TIMEOUT
    finally:
        nv.debug_inject(nv.INJECT_WAIT_TIMEOUT, 0)
    again = nv.decompress(m, nv.FP16)
    assert torch.equal(again[0], ref[0]) and torch.equal(again[1], ref[1])
    nv.mlp_grad(m, 2, pts, tgt, 0, nv.BF16)      # no timeout left behind


def test_allocation_budget(model):
    g, m = model
    ijk, val, _ = workload("sphere32")
    nv.debug_inject(nv.INJECT_ALLOC_BUDGET, 1 << 16)
    try:
        with pytest.raises(nv.NvdbError) as e:
            nv.compress(g, steps=2, batch=1024)
        assert e.value.status == OOM
        with pytest.raises(nv.NvdbError) as e:
            nv.build(ijk.cuda().contiguous(), val.cuda().contiguous(), 0, 3.0)
        assert e.value.status == OOM
    finally:
        nv.debug_inject(nv.INJECT_ALLOC_BUDGET, 0)
    again = nv.compress(g, seed=1, ffm_sigma=1.0, steps=20, batch=1024)
    assert again.export() == m.export()
    with pytest.raises(nv.NvdbError) as e:
        nv.debug_inject(99, 0)
    assert e.value.status == 1
