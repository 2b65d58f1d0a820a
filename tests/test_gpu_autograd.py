"""The networks as a torch.autograd.Function (Section 3.2): forward through the network
kernel, backward through the hand-written gradient kernel with the upstream dL/dy as a
linear loss; training with a torch optimiser, then re-patching and decoding."""
import numpy as np
import pytest
import torch

import paper_2208_04448_b300 as nv
from fixtures import workload
from gpu_helpers import bf16_weight_sensitivity, oracle_forward_scale, randomise_biases, rel_err
from oracle import blob, codec, vdb
from oracle import nets as N

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sphere():
    ijk, val, _ = workload("sphere128")
    ijk, val = ijk.numpy(), val.numpy()
    return ijk, val, vdb.build(ijk, val)


def _cuda(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def _imported(ref, seed):
    opts = codec.default_opts(seed=seed, sigma=1.25, width=[32, 64, 64], layers=[3, 4, 4])
    opts["ffm_size"] = [32, 64]
    om = randomise_biases(codec.init_model(ref, 0, 3.0, opts), seed)
    codec.make_patches(ref, om)
    return om, nv.model_import(blob.write(om))


@pytest.mark.parametrize("net", [0, 1, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_autograd_gradient_matches_oracle(sphere, net, prec):
    ijk, val, ref = sphere
    om, m = _imported(ref, 21)
    r = np.random.default_rng(net)
    pts = ref["ijk"][r.integers(0, ref["n"], 3000)].astype(np.int32)
    if net == 0:
        pts = pts >> 3 << 3   # the level-1 classifier sees leaf units either way
    w = r.standard_normal(len(pts)).astype(np.float32).astype(np.float64)
    params = m.params(net).clone().requires_grad_(True)
    y = nv.network(params, m, net, _cuda(pts, torch.int32), prec)
    (y * _cuda(w, torch.float32)).sum().backward()
    y_ref, cache = N.forward(om["nets"][net], N.encode(codec.level_coords(om, net, pts), codec.level_q(om, net)))
    g_ref = N.flatten(N.backward(om["nets"][net], cache, w))
    g = params.grad.cpu().numpy()
    want, scale = oracle_forward_scale(om, net, pts)
    if prec == 0:
        assert rel_err(y.detach().cpu().numpy(), want, scale).max() <= 1e-5
        assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    else:   # BF16 operands: within 3x what rounding the weights alone to BF16 moves (+ u)
        z = N.encode(codec.level_coords(om, net, pts), codec.level_q(om, net))
        g_sens = bf16_weight_sensitivity(om["nets"][net], z, lambda yb: w)
        nref = np.linalg.norm(g_ref)
        assert np.linalg.norm(g - g_ref) / nref <= 3.0 * np.linalg.norm(g_sens - g_ref) / nref + 2.0 ** -9


def test_torch_optimiser_trains_then_repatch_and_decode(sphere):
    ijk, val, ref = sphere
    g = nv.build(_cuda(ijk, torch.int32), _cuda(val, torch.float32), 0, 3.0)
    m = nv.compress(g, seed=3, ffm_sigma=1.25, steps=0, patch_precs=1)
    params = m.params(nv.NET_REGRESSOR).clone().requires_grad_(True)
    opt = torch.optim.Adam([params], lr=1e-3)
    vox, tgt = _cuda(ref["ijk"], torch.int32), _cuda(ref["val"] / 3.0, torch.float32)
    gen = torch.Generator(device="cuda").manual_seed(0)
    losses = []
    for _ in range(150):
        idx = torch.randint(0, vox.shape[0], (4096,), device="cuda", generator=gen)
        y = nv.network(params, m, nv.NET_REGRESSOR, vox[idx].contiguous())
        loss = ((y - tgt[idx]) ** 2).mean()
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert np.mean(losses[-10:]) < 0.3 * np.mean(losses[:10])
    m.set_params(nv.NET_REGRESSOR, params.detach())
    with pytest.raises(nv.NvdbError) as e:          # the patches belonged to the old weights
        nv.decompress(m, nv.FP32)
    assert e.value.status == 7
    m.repatch(g, 1 << nv.FP32)
    dijk, dval, cnt = nv.decompress(m, nv.FP32)
    assert cnt == [ref["n"]] and np.array_equal(dijk.cpu().numpy(), ref["ijk"])
    om = blob.read(m.export())
    assert np.array_equal(N.flatten(om["nets"][2]), params.detach().cpu().numpy().astype(np.float64))
    want, scale = oracle_forward_scale(om, codec.REG, ref["ijk"])
    assert rel_err(dval.cpu().numpy() / 3.0, want, scale).max() <= 1e-5


def test_parameter_and_repatch_errors(sphere):
    ijk, val, ref = sphere
    g = nv.build(_cuda(ijk, torch.int32), _cuda(val, torch.float32), 0, 3.0)
    m = nv.compress(g, seed=3, steps=0, patch_precs=1)
    with pytest.raises(ValueError):
        m.set_params(0, torch.zeros(5, device="cuda"))
    other = nv.build(_cuda(ijk[: len(ijk) // 2], torch.int32), _cuda(val[: len(val) // 2], torch.float32), 0, 3.0)
    with pytest.raises(nv.NvdbError) as e:
        m.repatch(other, 1)
    assert e.value.status == 1
    with pytest.raises(ValueError):
        nv.network(m.params(2).requires_grad_(True), m, 2, _cuda(ref["ijk"][:10], torch.int32), nv.FP16)
