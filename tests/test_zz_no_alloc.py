"""nvdb_mlp_grad_static, the gradient entry point that allocates no device memory.

It is for callers that may not call cudaMalloc/cudaFree themselves or through
the library: applications that hand all device memory out of their own pool,
and latency-critical loops that cannot afford an allocation or the device-wide
synchronisation a free can cause.  It must give the gradient and loss of
nvdb_mlp_grad (summation order aside), call after call, and leave the free
device memory unchanged.

This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

import paper_2208_04448_b300 as nv
from fixtures import workload
from oracle import blob, codec, vdb

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4   # the FP32 gradient bar of the parity tests


def _model():
    ijk, val, _ = workload("sphere32")
    g = vdb.build(ijk.numpy(), val.numpy())
    om = codec.init_model(g, 0, 3.0, codec.default_opts(seed=21, sigma=1.0, width=[32, 64, 64], layers=[3, 4, 4],
                                                        ffm_size=[32, 64]))
    codec.make_patches(g, om)
    return g, nv.model_import(blob.write(om))


def test_static_gradient_matches_allocating_entry_point_twice():
    g, m = _model()
    r = np.random.default_rng(5)
    cases = []
    for net, loss in ((2, nv.LOSS_MSE), (1, nv.LOSS_BCE), (0, nv.LOSS_BCE)):
        n = 5000
        pts = torch.from_numpy(g["ijk"][r.integers(0, g["n"], n)].astype(np.int32)).cuda()
        tgt = torch.from_numpy((r.random(n) > 0.5).astype(np.float32) if loss == nv.LOSS_BCE
                               else r.standard_normal(n).astype(np.float32)).cuda()
        ref, lref = nv.mlp_grad(m, net, pts, tgt, loss)
        cases.append((net, loss, pts, tgt, ref.cpu().numpy(), lref))
    outs = [torch.empty(m.param_count(net), dtype=torch.float32, device="cuda") for net, *_ in cases]
    # One-time set-up outside the measured region: the first call on a device looks the static
    # array's address up, and torch loads its own fill kernel (a device-memory change of torch's).
    nv.mlp_grad_static(m, cases[0][0], cases[0][2], cases[0][3], cases[0][1], out=outs[0])
    outs[0].fill_(float("nan"))
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for call in range(2):                                   # two calls in a row of every case
        for (net, loss, pts, tgt, ref, lref), out in zip(cases, outs):
            out.fill_(float("nan"))
            got, lgot = nv.mlp_grad_static(m, net, pts, tgt, loss, out=out)
            got = got.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.abs(got - ref).max() <= GRAD_TOL * np.abs(ref).max(), (call, net)
            assert abs(lgot - lref) <= 1e-5 * max(1.0, abs(lref)), (call, net)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free_before) < (2 << 20)
    # A cudaMalloc / cudaFree pair inside a call would leave the free memory unchanged: run
    # the calls again with a one-byte allocation budget, under which any library allocation
    # fails (NVDB_ERR_OUT_OF_MEMORY), and check that they still succeed and agree.
    nv.debug_inject(nv.INJECT_ALLOC_BUDGET, 1)
    try:
        for (net, loss, pts, tgt, ref, lref), out in zip(cases, outs):
            out.fill_(float("nan"))
            got, lgot = nv.mlp_grad_static(m, net, pts, tgt, loss, out=out)
            assert np.abs(got.cpu().numpy() - ref).max() <= GRAD_TOL * np.abs(ref).max(), net
            assert abs(lgot - lref) <= 1e-5 * max(1.0, abs(lref)), net
        with pytest.raises(nv.NvdbError):   # the allocating entry point does fail under it
            nv.mlp_grad(m, cases[0][0], cases[0][2], cases[0][3], cases[0][1])
    finally:
        nv.debug_inject(nv.INJECT_ALLOC_BUDGET, 0)


def test_static_gradient_capacity_error():
    """Networks whose partials do not fit the static array are rejected with CAPACITY (the
    limit is lowered below one partial of the network, since no supported shape reaches
    2^20 - 2 parameters), and a fitting limit with a single partial slot still agrees."""
    g, m = _model()
    r = np.random.default_rng(9)
    n = 3000
    pts = torch.from_numpy(g["ijk"][r.integers(0, g["n"], n)].astype(np.int32)).cuda()
    tgt = torch.from_numpy(r.standard_normal(n).astype(np.float32)).cuda()
    P = m.param_count(2)
    ref, lref = nv.mlp_grad(m, 2, pts, tgt, nv.LOSS_MSE)
    try:
        nv.debug_inject(nv.INJECT_STATIC_LIMIT, P + 1)
        with pytest.raises(nv.NvdbError) as e:
            nv.mlp_grad_static(m, 2, pts, tgt, nv.LOSS_MSE)
        assert e.value.status == nv.ERR_CAPACITY
        nv.debug_inject(nv.INJECT_STATIC_LIMIT, P + 2)   # room for exactly one block's partial
        got, lgot = nv.mlp_grad_static(m, 2, pts, tgt, nv.LOSS_MSE)
        ref = ref.cpu().numpy()
        assert np.abs(got.cpu().numpy() - ref).max() <= GRAD_TOL * np.abs(ref).max()
        assert abs(lgot - lref) <= 1e-5 * max(1.0, abs(lref))
    finally:
        nv.debug_inject(nv.INJECT_STATIC_LIMIT, 0)
