"""Checkpoint / resume: a compress that continues an interrupted one (its master weights,
Adam moments and step count; Philox batches and the learning-rate schedule are keyed by
the global step) equals the uninterrupted run bit for bit."""
import numpy as np
import pytest
import torch

import paper_2208_04448_b300 as nv
from fixtures import workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_resume_equals_uninterrupted(prec):
    ijk, val, _ = workload("union128")
    g = nv.build(ijk.cuda().contiguous(), val.cuda().contiguous(), 0, 3.0)
    kw = dict(seed=5, ffm_sigma=1.25, batch=4096, train_prec=prec, patch_precs=1)
    full = nv.compress(g, steps=130, **kw)                   # crosses the decay at step 101
    first = nv.compress(g, steps=70, **kw)
    rest = nv.compress(g, steps=60, warm=first, resume=1, **kw)
    for k in range(3):
        assert len(rest.losses(k)) == 130
        assert np.array_equal(rest.losses(k), full.losses(k))
    assert rest.export() == full.export()
    # a warm start (no resume) restarts Adam and the step count: a different run
    warm = nv.compress(g, steps=60, warm=first, **kw)
    assert len(warm.losses(0)) == 60 and warm.export() != full.export()
