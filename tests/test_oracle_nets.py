"""Pins of the oracle's encoding, MLP, losses, gradients and Adam (CPU only)."""
import math

import numpy as np
import pytest

from oracle import nets as N
from oracle import rng


def test_encoding_at_origin_is_cos1_sin0():
    q = rng.ffm_increments(5, 0, 16, 10.0, 1024)
    z = N.encode(np.zeros((1, 3), np.int64), q)
    assert np.array_equal(z[0, :16], np.ones(16)) and np.array_equal(z[0, 16:], np.zeros(16))


def test_encoding_lattice_shift_is_complex_rotation():
    q = rng.ffm_increments(5, 0, 16, 10.0, 1024)
    r = np.random.default_rng(0)
    c = r.integers(0, 1 << 20, (50, 3))
    for d in range(3):
        e = np.zeros(3, np.int64); e[d] = 1
        z0, z1 = N.encode(c, q), N.encode(c + e, q)
        a = z0[:, :16] + 1j * z0[:, 16:]
        b = z1[:, :16] + 1j * z1[:, 16:]
        s = q[:, d].astype(np.int64)
        s = np.where(s >= 1 << 31, s - (1 << 32), s)
        rot = np.exp(2j * np.pi * s / 2.0 ** 32)
        assert np.max(np.abs(b - a * rot[None])) < 1e-9


def test_encoding_equals_fourier_features_of_normalised_coords():
    # gamma = [cos 2 pi B x, sin 2 pi B x], x = c / E, B = q E / 2^32 (q as signed)
    E = 512
    q = rng.ffm_increments(11, 0, 8, 2.0, E)
    s = q.astype(np.int64)
    B = np.where(s >= 1 << 31, s - (1 << 32), s) * E / 2.0 ** 32
    c = np.random.default_rng(1).integers(0, E, (100, 3))
    x = c / E
    ang = 2 * np.pi * x @ B.T
    want = np.concatenate([np.cos(ang), np.sin(ang)], 1)
    assert np.max(np.abs(N.encode(c, q) - want)) < 1e-9


HAND_NET = dict(W=[np.array([[1.0, -2.0], [0.5, 1.0]]), np.array([[2.0, 1.0], [-1.0, 3.0]])],
                b=[np.array([0.5, -1.0]), np.array([0.0, 0.25])],
                wh=np.array([1.5, -2.0]), bh=0.1)


def test_forward_hand_expanded():
    # z=(1,2): a1=(1-4+.5, .5+2-1)=(-2.5,1.5) h1=(0,1.5); a2=(1.5, 4.5+.25) ; y=2.25-9.5+.1
    # z=(-1,.5): a1=(-1.5,-1) h1=0; a2=(0,.25); y=-.5+.1
    y, (hs, pre) = N.forward(HAND_NET, np.array([[1.0, 2.0], [-1.0, 0.5]]))
    assert np.allclose(pre[0], [[-2.5, 1.5], [-1.5, -1.0]], atol=0, rtol=0)
    assert np.allclose(hs[2], [[1.5, 4.75], [0.0, 0.25]], atol=0, rtol=0)
    assert y[0] == pytest.approx(-7.15, abs=1e-14) and y[1] == pytest.approx(-0.4, abs=1e-14)


def test_losses_closed_forms():
    l, g = N.loss_and_grad(np.zeros(4), np.array([0, 1, 0, 1.0]), N.LOSS_BCE)
    assert l == pytest.approx(math.log(2.0), abs=1e-15)
    assert np.allclose(g, np.array([0.5, -0.5, 0.5, -0.5]) / 4, atol=1e-16)
    l, g = N.loss_and_grad(np.array([100.0, -100.0]), np.array([1.0, 1.0]), N.LOSS_BCE)
    assert l == pytest.approx(50.0, abs=1e-12)
    assert g[0] == pytest.approx(0.0, abs=1e-40) and g[1] == pytest.approx(-0.5, abs=1e-40)
    l, g = N.loss_and_grad(np.array([1.0, 3.0]), np.array([0.0, 1.0]), N.LOSS_MSE)
    assert l == 2.5 and np.array_equal(g, [1.0, 2.0])
    l, g = N.loss_and_grad(np.array([1.0, 3.0, 2.0]), np.array([2.0, 1.0, 2.0]), N.LOSS_L1)
    assert l == 1.0 and np.array_equal(g, [-1.0 / 3, 1.0 / 3, 0.0])


@pytest.mark.parametrize("kind", [N.LOSS_BCE, N.LOSS_MSE, N.LOSS_L1])
def test_backward_matches_central_differences(kind):
    r = np.random.default_rng(kind)
    net = rng.xavier_net(seed=77, net=kind, n_in=6, width=5, layers=3)
    net["b"] = [r.standard_normal(5) * 0.1 for _ in range(3)]
    net["bh"] = 0.05
    z = r.standard_normal((40, 6))
    y, cache = N.forward(net, z)
    keep = np.all([np.all(np.abs(a) > 1e-3, axis=1) for a in cache[1]], axis=0)
    z = z[keep]
    t = (r.random(z.shape[0]) > 0.5).astype(float) if kind == N.LOSS_BCE else r.standard_normal(z.shape[0])
    if kind == N.LOSS_L1:
        t = N.forward(net, z)[0] + np.where(r.random(z.shape[0]) > 0.5, 0.3, -0.3)
    y, cache = N.forward(net, z)
    _, g = N.loss_and_grad(y, t, kind)
    ana = N.flatten(N.backward(net, cache, g))
    theta = N.flatten(net)
    num = np.zeros_like(theta)
    for i in range(theta.size):
        h = 1e-6 * max(1.0, abs(theta[i]))
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h; tm[i] -= h
        lp = N.loss_and_grad(N.forward(N.unflatten(tp, net), z)[0], t, kind)[0]
        lm = N.loss_and_grad(N.forward(N.unflatten(tm, net), z)[0], t, kind)[0]
        num[i] = (lp - lm) / (2 * h)
    assert np.max(np.abs(ana - num)) <= 1e-6 * max(1.0, np.max(np.abs(num)))


def test_adam_first_and_second_step_closed_form():
    g1 = np.array([0.3, -2.0, 1e-9, 0.0])
    th = np.array([1.0, 1.0, 1.0, 1.0])
    m, v = np.zeros(4), np.zeros(4)
    N.adam_step(th, m, v, g1.copy(), 1, 1e-3)
    assert np.allclose(th, 1.0 - 1e-3 * g1 / (np.abs(g1) + 1e-8), rtol=0, atol=1e-15)
    g2 = np.array([0.1, 0.5, -1.0, 2.0])
    th2 = th.copy()
    N.adam_step(th2, m, v, g2.copy(), 2, 5e-4)
    mh = (0.1 * (0.9 * g1 + g2)) / (1 - 0.9 ** 2)
    vh = (0.001 * (0.999 * g1 ** 2 + g2 ** 2)) / (1 - 0.999 ** 2)
    assert np.allclose(th2, th - 5e-4 * mh / (np.sqrt(vh) + 1e-8), rtol=0, atol=1e-15)


def test_lr_schedule():
    assert N.lr_at(1, 1e-3, 0.975, 100) == 1e-3
    assert N.lr_at(100, 1e-3, 0.975, 100) == 1e-3
    assert N.lr_at(101, 1e-3, 0.975, 100) == pytest.approx(0.975e-3)
    assert N.lr_at(250, 1e-3, 0.5, 100) == pytest.approx(0.25e-3)
    assert N.lr_at(9999, 1e-3, 0.5, 0) == 1e-3


def test_flatten_order():
    v = N.flatten(HAND_NET)
    assert np.array_equal(v, [1, -2, 0.5, 1, 0.5, -1, 2, 1, -1, 3, 0, 0.25, 1.5, -2, 0.1])
    back = N.unflatten(v, HAND_NET)
    assert all(np.array_equal(a, b) for a, b in zip(back["W"], HAND_NET["W"]))
