"""The arithmetic each tensor-core precision specifies, computed in FP64 (test infrastructure).

The paper leaves precision open (it names mixed precision as future work, Section 5); the
decode kernels state theirs, and this module follows those statements, not the kernels'
code:

  operands   rounded from FP32 to the precision's format (round to nearest even): FP16,
             BF16, or E4M3 with saturation to +-448 (subnormal spacing 2^-9);
  products   summed exactly (FP64 here, FP32 in tensor memory on the GPU);
  bias       added in FP32 after the sum (FP16: it enters the sum as the pair
             fp16(b) + fp16(b - fp16(b))); ReLU; the next layer's operand is rounded again;
  head       an FP32 dot product on the last hidden layer's ReLU output (one per class for
             the ternary level-1 classifier).
  sin        networks with the sin activation (16-bit modes only) take h = f32(sin(f32(omega a)))
             on the FP32 pre-activation a in place of the ReLU (the kernels use the MUFU sine,
             whose error sits far inside the parity bar).

  FP16     every operand FP16.
  BF16     the encoding and the inputs of every hidden layer except the last carried as a
           pair hi = bf16(v), lo = bf16(v - hi); products hi*W_hi + lo*W_hi, plus hi*W_lo
           when the weights are not BF16 values (W_hi = bf16(W), W_lo = bf16(W - W_hi)).
  BF16X3   as BF16 with every hidden layer's input carried as a pair.
  FP8      layer 0 as FP16 on the encoding; hidden layer l >= 1 takes E4M3 activations
           q = e4m3(relu(h) / s_l) and E4M3 weights e4m3(W_l / s_w,l), s_w,l = max|W_l| / 448;
           every layer's epilogue is h = alpha_l D + beta_l with
             l = 0:          alpha = 1 / s_1,              beta = b_0 / s_1
             0 < l < L-1:    alpha = s_w,l s_l / s_{l+1},   beta = b_l / s_{l+1}
             l = L-1 > 0:    alpha = s_w,l s_l,             beta = b_l
           (alpha = 1, beta = b_0 when L = 1).  The activation ranges a_l = 448 s_l are
           min(16 amax_l, bound_l): amax_l the largest ReLU output of layer l-1 over 2^12
           points of the network's domain drawn from the SplitMix64 stream of seed
           0xF8CA11B (draw s: coordinates (z & m, (z >> 21) & m, (z >> 42) & m), m = extent - 1
           in the level's units), bound_l = max_o sum_i |W_{l-1}[o, i]| a_{l-1} + |b_{l-1}[o]|
           with a_0 = 1 (the encoding is bounded by 1).

This is an independent restatement: it shares no code with the CUDA path, and no value in
it comes from the GPU.  A kernel that matches it element by element computes what its
precision promises; how far that promise is from the unrounded network is a separate,
reported measurement.
"""
from __future__ import annotations

import numpy as np

from . import nets as N

PREC_FP32, PREC_BF16, PREC_FP8, PREC_FP16, PREC_BF16X3 = 0, 1, 2, 3, 4
FP8_CALIB_SEED = 0xF8CA11B
FP8_CALIB_POINTS = 1 << 12
FP8_HEADROOM = 16.0   # measured activation range = FP8_HEADROOM x the calibration amax (capped by the bound)
E4M3_MAX = 448.0


def f32(x):
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float64)


def bf16(x):
    """FP32 -> BF16, round to nearest even, as float64."""
    u = np.asarray(x, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def f16(x):
    """FP32 -> FP16, round to nearest even, as float64."""
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float16).astype(np.float64)


def e4m3(x):
    """FP32 -> E4M3 (4 exponent bits, bias 7; 3 mantissa bits; no infinities), round to
    nearest even, saturating to +-448; as float64."""
    x = np.asarray(x, np.float64).astype(np.float32).astype(np.float64)
    a = np.minimum(np.abs(x), E4M3_MAX)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -9)))
    e = np.maximum(e, -6.0)                  # below 2^-6 the spacing stays 2^-9 (subnormals)
    step = 2.0 ** (e - 3)
    q = np.round(a / step) * step            # numpy rounds halves to even
    return np.sign(x) * np.minimum(q, E4M3_MAX)


def split_bf16(x):
    hi = bf16(x)
    return hi, bf16(f32(f32(x) - hi))


def _mix64(z):
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def calib_coords(log2_extent: int, n: int = FP8_CALIB_POINTS, seed: int = FP8_CALIB_SEED) -> np.ndarray:
    """The FP8 calibration points (level units, relative to the domain origin)."""
    s = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix64(np.uint64(seed) + np.uint64(0x9E3779B97F4A7C15) * s)
    m = np.uint64((1 << log2_extent) - 1)
    return np.stack([z & m, (z >> np.uint64(21)) & m, (z >> np.uint64(42)) & m], -1).astype(np.int64)


def fp8_epilogue(net: dict, q: np.ndarray, log2_extent: int):
    """(alpha_l, beta_l[W], s_w,l, s_l) per layer, following the definition above."""
    L = len(net["W"])
    z = N.encode(calib_coords(log2_extent), q)
    _, (hs, _) = N.forward(net, z)
    amax = [float(np.max(hs[l + 1])) for l in range(L)]          # ReLU output of layer l
    a_in = 1.0
    out = []
    for l in range(L):
        W, b = net["W"][l], net["b"][l]
        bound = float(np.max(np.abs(W).sum(1) * a_in + np.abs(b)))
        meas = FP8_HEADROOM * amax[l] if l < L - 1 else 0.0
        a_out = min(meas, bound) if meas > 0 else (bound if bound > 0 else 1.0)
        s_in, s_out = a_in / E4M3_MAX, a_out / E4M3_MAX
        s_w = float(np.max(np.abs(W))) / E4M3_MAX if np.max(np.abs(W)) > 0 else 1.0
        if l == 0:
            alpha = 1.0 / s_out if L > 1 else 1.0
            beta = b * alpha
        elif l < L - 1:
            alpha, beta = s_w * s_in / s_out, b / s_out
        else:
            alpha, beta = s_w * s_in, b
        out.append((alpha, np.asarray(beta, np.float64), s_w, s_in))
        a_in = a_out
    return out


def _bf16_exact(net: dict) -> bool:
    return all(np.array_equal(bf16(W), W) for W in net["W"]) and all(np.array_equal(bf16(b), b) for b in net["b"])


def forward(net: dict, z: np.ndarray, prec: int, q=None, log2_extent=None) -> np.ndarray:
    """Network output y [N] at encoded inputs z [N, n] in the arithmetic of `prec`.
    FP8 needs the level's Fourier matrix q and extent (for the calibration points)."""
    L = len(net["W"])
    z = f32(z)
    if prec == PREC_FP8:
        ep = fp8_epilogue(net, q, log2_extent)
        a = f16(z) @ f16(net["W"][0]).T
        for l in range(L):
            alpha, beta, s_w, _ = ep[l]
            if l > 0:
                a = hq @ e4m3(f32(net["W"][l] / s_w)).T
            pre = alpha * a + beta
            if l < L - 1:
                hq = e4m3(np.maximum(pre, 0.0))
            else:
                h = np.maximum(f32(pre), 0.0)
        return _head(net, h)
    exact = _bf16_exact(net)
    sin = net.get("act", 0) == 1
    if sin and prec == PREC_FP8:
        raise ValueError("sin networks: 16-bit precisions only")

    def act(a):
        a = f32(a)
        return f32(np.sin(f32(net["omega"] * a))) if sin else np.maximum(a, 0.0)
    h = z
    for l, (W, b) in enumerate(zip(net["W"], net["b"])):
        if prec == PREC_FP16:
            bh = f16(b)
            a = f16(h) @ f16(W).T + bh + f16(f32(f32(b) - bh))
            h = act(a)
            continue
        else:
            comp = prec == PREC_BF16X3 or l < L - 1
            hh, hl = split_bf16(h)
            wh, wl = split_bf16(W)
            a = hh @ wh.T
            if comp:
                a = a + hl @ wh.T
            if not exact:
                a = a + hh @ wl.T
        h = act(f32(a) + b)
    return _head(net, h)


def _head(net: dict, h: np.ndarray) -> np.ndarray:
    wh = np.asarray(net["wh"], dtype=np.float64)
    return h @ (wh.T if wh.ndim == 2 else wh) + net["bh"]
