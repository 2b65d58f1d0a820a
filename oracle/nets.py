"""Encoding, MLP forward/backward, losses and Adam in FP64.

Encoding (Section 3.2.2, Eq. 2, with the Fourier feature mapping of Tancik
et al. that the paper adopts): for integer coordinates c (relative to the
domain origin, in the level's units) and the level's fixed-point Fourier
matrix q (uint32 [m, 3]),
    Phi_f = sum_d q[f, d] * c_d  mod 2^32            (exact integer phase)
    gamma(c) = [cos(2 pi Phi_f / 2^32)]_f ++ [sin(2 pi Phi_f / 2^32)]_f,
which equals [cos 2 pi B x, sin 2 pi B x] with x = c / E and B = q E / 2^32.

Networks (Section 3.2, Section 3.3.1): `layers` hidden layers
h_{l+1} = act(W_l h_l + b_l) followed by a linear head y = W_h h_L + b_h with one
output (w_h a vector, b_h a scalar) or C outputs (W_h [C][width], b_h [C]).  The
activation (Appendix "Effect of Activation Functions" and the hyper-parameter table's
Activation/Freq. column) is ReLU (ReLU'(0) = 0) or sin with frequency omega:
act(a) = sin(omega a), act'(a) = omega cos(omega a).  A binary classifier's y is
the logit (active iff y > 0); the ternary level-1 classifier's three outputs are
class logits (the class is the first maximum); a regressor's y is the value.

Losses, each the mean over the batch: MSE (Eq. 1), binary cross-entropy with
logits for the level-0 mask, cross-entropy over softmax for the ternary level-1
mask (Section 3.3.1), and L1.
Adam (Kingma & Ba 2014; Section 3.2) with beta1 = 0.9, beta2 = 0.999,
eps = 1e-8, bias correction, and learning rate lr * gamma^floor((t-1)/interval)
(exponential decay, Section 3.2 and the hyper-parameter table).
"""
from __future__ import annotations

import numpy as np

LOSS_MSE, LOSS_L1, LOSS_BCE, LOSS_CE = 0, 1, 2, 3
ACT_RELU, ACT_SIN = 0, 1
BETA1, BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


def phase(c: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Exact fixed-point phases Phi [N, m] (uint64 holding values < 2^32)."""
    c = np.asarray(c, dtype=np.int64).astype(np.uint64)       # two's complement wrap is exact mod 2^32
    q = np.asarray(q, dtype=np.uint64)
    with np.errstate(over="ignore"):
        p = (c[:, None, :] * q[None, :, :]).sum(-1)
    return p & np.uint64(0xFFFFFFFF)


def encode(c: np.ndarray, q: np.ndarray) -> np.ndarray:
    """gamma(c) [N, 2m] in FP64."""
    p = phase(c, q).astype(np.int64)
    p = np.where(p >= (1 << 31), p - (1 << 32), p).astype(np.float64)
    ang = (2.0 * np.pi / 4294967296.0) * p
    return np.concatenate([np.cos(ang), np.sin(ang)], axis=1)


def act(net: dict, a: np.ndarray) -> np.ndarray:
    if net.get("act", ACT_RELU) == ACT_SIN:
        return np.sin(net["omega"] * a)
    return np.maximum(a, 0.0)


def act_grad(net: dict, a: np.ndarray) -> np.ndarray:
    if net.get("act", ACT_RELU) == ACT_SIN:
        return net["omega"] * np.cos(net["omega"] * a)
    return (a > 0).astype(np.float64)


def forward(net: dict, z: np.ndarray):
    """Returns (y [N] or [N, C], cache) with cache = (h_0..h_L, a_1..a_L)."""
    hs, pre = [np.asarray(z, dtype=np.float64)], []
    for W, b in zip(net["W"], net["b"]):
        a = hs[-1] @ W.T + b
        pre.append(a)
        hs.append(act(net, a))
    wh = np.asarray(net["wh"], dtype=np.float64)
    y = hs[-1] @ (wh.T if wh.ndim == 2 else wh) + net["bh"]
    return y, (hs, pre)


def classify3(y: np.ndarray) -> np.ndarray:
    """Class of each row of three logits: the first maximum (ties go to the lower class)."""
    return np.argmax(np.asarray(y), axis=1)


def loss_and_grad(y: np.ndarray, t: np.ndarray, kind: int):
    """Mean loss over the batch and dL/dy."""
    y = np.asarray(y, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    n = y.shape[0]
    if kind == LOSS_CE:                        # t: class indices; y: [N, C] logits
        lab = np.asarray(t, dtype=np.int64)
        mx = y.max(1, keepdims=True)
        lse = mx[:, 0] + np.log(np.exp(y - mx).sum(1))
        l = lse - y[np.arange(n), lab]
        g = np.exp(y - lse[:, None])
        g[np.arange(n), lab] -= 1.0
        return float(l.mean()), g / n
    if kind == LOSS_BCE:
        l = np.maximum(y, 0.0) - y * t + np.log1p(np.exp(-np.abs(y)))
        g = (1.0 / (1.0 + np.exp(-y)) - t) / n
    elif kind == LOSS_MSE:
        l = (y - t) ** 2
        g = 2.0 * (y - t) / n
    elif kind == LOSS_L1:
        l = np.abs(y - t)
        g = np.sign(y - t) / n
    else:
        raise ValueError(kind)
    return float(l.mean()), g


def backward(net: dict, cache, g: np.ndarray) -> dict:
    """Gradients of the mean loss w.r.t. every parameter, given dL/dy = g ([N] or [N, C])."""
    hs, pre = cache
    L = len(net["W"])
    grads = dict(W=[None] * L, b=[None] * L)
    wh = np.asarray(net["wh"], dtype=np.float64)
    if wh.ndim == 2:
        grads["wh"] = g.T @ hs[L]
        grads["bh"] = g.sum(0)
        delta = (g @ wh) * act_grad(net, pre[L - 1])
    else:
        grads["wh"] = hs[L].T @ g
        grads["bh"] = float(g.sum())
        delta = np.outer(g, wh) * act_grad(net, pre[L - 1])
    for l in range(L - 1, -1, -1):
        grads["W"][l] = delta.T @ hs[l]
        grads["b"][l] = delta.sum(0)
        if l > 0:
            delta = (delta @ net["W"][l]) * act_grad(net, pre[l - 1])
    return grads


def flatten(p: dict) -> np.ndarray:
    """Parameter vector in storage order: W_0, b_0, ..., W_{L-1}, b_{L-1}, W_h (row-major), b_h."""
    parts = []
    for W, b in zip(p["W"], p["b"]):
        parts += [np.asarray(W, dtype=np.float64).reshape(-1), np.asarray(b, dtype=np.float64).reshape(-1)]
    parts += [np.asarray(p["wh"], dtype=np.float64).reshape(-1), np.asarray(p["bh"], dtype=np.float64).reshape(-1)]
    return np.concatenate(parts)


def unflatten(v: np.ndarray, like: dict) -> dict:
    out = {k: like[k] for k in ("act", "omega") if k in like}
    out.update(W=[], b=[])
    o = 0
    for W, b in zip(like["W"], like["b"]):
        out["W"].append(v[o:o + W.size].reshape(W.shape)); o += W.size
        out["b"].append(v[o:o + b.size].reshape(b.shape)); o += b.size
    wh = np.asarray(like["wh"])
    out["wh"] = v[o:o + wh.size].reshape(wh.shape).copy(); o += wh.size
    out["bh"] = float(v[o]) if wh.ndim == 1 else v[o:o + wh.shape[0]].copy()
    return out


def lr_at(step: int, lr: float, decay: float, interval: int) -> float:
    """Learning rate of step t (1-based): lr * decay^floor((t-1)/interval); constant if interval == 0."""
    if interval <= 0:
        return lr
    return lr * decay ** ((step - 1) // interval)


def adam_step(theta: np.ndarray, m: np.ndarray, v: np.ndarray, g: np.ndarray, step: int, lr_t: float):
    """One Adam update (in place on theta, m, v)."""
    m *= BETA1
    m += (1.0 - BETA1) * g
    v *= BETA2
    v += (1.0 - BETA2) * g * g
    mhat = m / (1.0 - BETA1 ** step)
    vhat = v / (1.0 - BETA2 ** step)
    theta -= lr_t * mhat / (np.sqrt(vhat) + ADAM_EPS)
