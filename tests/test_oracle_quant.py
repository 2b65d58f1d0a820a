"""Pins of oracle/quant.py, the FP64 statement of the tensor-core precisions (CPU only).

The rounding functions are pinned by values fixed by the formats' definitions (IEEE
binary16, bfloat16 = the upper half of binary32, OCP E4M3: bias 7, 3 mantissa bits,
largest finite 448, subnormal spacing 2^-9); the quantised forward passes by networks
whose every operand is exactly representable (they must equal the FP64 forward) and by
a hand-expanded two-layer FP8 example.
"""
import numpy as np
import pytest

from oracle import nets as N
from oracle import quant as Q


def test_e4m3_values():
    x = np.array([0.0, 1.0, 448.0, 500.0, -500.0, 1.0625, 1.1875, 1.125, 0.5, 2.0 ** -6, 2.0 ** -9,
                  1.5 * 2.0 ** -9, 2.0 ** -10, 3.0 * 2.0 ** -11, 240.0, 232.0, 248.0, -1.3])
    want = np.array([0.0, 1.0, 448.0, 448.0, -448.0, 1.0, 1.25, 1.125, 0.5, 2.0 ** -6, 2.0 ** -9,
                     2.0 * 2.0 ** -9, 0.0, 2.0 ** -9, 240.0, 224.0, 256.0, -1.25])
    assert np.array_equal(Q.e4m3(x), want)
    # the 126 finite positive values: 7 subnormals k 2^-9, then (1 + m/8) 2^e for e = -6..8
    # (without 1.875 * 2^8 = 480, the NaN code); each maps to itself, and every value in
    # between rounds to one of its two neighbours (halves to the even mantissa)
    vals = [k * 2.0 ** -9 for k in range(1, 8)] + [(1 + m / 8) * 2.0 ** e for e in range(-6, 9) for m in range(8)]
    vals = np.array(sorted(v for v in vals if v <= 448.0))
    assert len(vals) == 126 and vals[-1] == 448.0
    assert np.array_equal(Q.e4m3(vals), vals)
    mid = (vals[:-1] + vals[1:]) / 2
    r = Q.e4m3(mid)
    assert np.all((r == vals[:-1]) | (r == vals[1:]))
    below = np.nextafter(mid.astype(np.float32), np.float32(0)).astype(np.float64)   # inputs are FP32
    above = np.nextafter(mid.astype(np.float32), np.float32(1e9)).astype(np.float64)
    assert np.array_equal(Q.e4m3(below), vals[:-1]) and np.array_equal(Q.e4m3(above), vals[1:])


def test_bf16_and_f16_values():
    # bf16 keeps 8 significant bits: 1 + 2^-8 is a tie (-> 1, even), 1 + 3 * 2^-8 rounds up
    x = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -7, -3.0, 65504.0])
    assert np.array_equal(Q.bf16(x), [1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -3.0, 65536.0])
    # f16 keeps 11 significant bits and saturates to inf past 65520
    y = np.array([1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 65504.0, 2.0 ** -24])
    assert np.array_equal(Q.f16(y), [1.0, 1.0 + 2.0 ** -9, 65504.0, 2.0 ** -24])
    r = np.random.default_rng(0).standard_normal(1000)
    hi, lo = Q.split_bf16(r)
    assert np.array_equal(Q.bf16(hi), hi) and np.array_equal(Q.bf16(lo), lo)
    assert np.all(np.abs(hi + lo - Q.f32(r)) <= 2.0 ** -16 * np.abs(r))


def _net(rng, nin, w, L, fmt):
    """A network whose weights and biases are exactly representable in `fmt`."""
    W = [fmt(rng.standard_normal((w, nin if l == 0 else w)) * 0.3) for l in range(L)]
    b = [fmt(rng.standard_normal(w) * 0.1) for _ in range(L)]
    return dict(W=W, b=b, wh=rng.standard_normal(w) * 0.5, bh=0.25)


@pytest.mark.parametrize("prec,fmt", [(Q.PREC_FP16, Q.f16), (Q.PREC_BF16, Q.bf16), (Q.PREC_BF16X3, Q.bf16)])
def test_representable_operands_are_exact(prec, fmt):
    """Inputs and weights exactly representable, and activations that stay so (a single
    hidden layer): the quantised forward equals the FP64 forward up to FP32 rounding."""
    rng = np.random.default_rng(3)
    net = _net(rng, 8, 8, 1, fmt)
    z = fmt(rng.uniform(-1, 1, (64, 8)))
    want, _ = N.forward(net, z)
    got = Q.forward(net, z, prec)
    assert np.allclose(got, want, rtol=1e-6, atol=1e-6)


def test_bf16_compensation_schedule():
    """BF16 carries every hidden input but the last as a hi + lo pair: with two layers the
    first layer sees the encoding to ~16 bits, the second a plain BF16 input.  Dropping
    the pair on the first layer (a plausible slip) moves the result by the encoding's
    rounding; BF16X3 keeps the pair on both."""
    rng = np.random.default_rng(4)
    net = _net(rng, 16, 16, 2, Q.bf16)
    z = rng.uniform(-1, 1, (256, 16))
    exact, cache = N.forward(net, z)
    h1 = cache[0][1]
    by_hand = np.maximum(Q.f32(Q.f32(Q.bf16(h1) @ net["W"][1].T) + net["b"][1]), 0) @ net["wh"] + net["bh"]
    got = Q.forward(net, z, Q.PREC_BF16)
    # equal except where the ~16-bit first layer puts h1 across a BF16 rounding boundary
    assert np.mean(np.abs(got - by_hand) > 1e-5) < 0.05
    assert np.allclose(Q.forward(net, z, Q.PREC_BF16X3), exact, rtol=0, atol=5e-5)
    assert np.abs(by_hand - exact).max() > 5e-4
    # a plain-BF16 encoding would move most rows
    h1_plain = np.maximum(Q.bf16(z) @ net["W"][0].T + net["b"][0], 0)
    plain = np.maximum(Q.bf16(h1_plain) @ net["W"][1].T + net["b"][1], 0) @ net["wh"] + net["bh"]
    assert np.mean(np.abs(got - plain) > 1e-5) > 0.5


def test_fp8_two_layer_by_hand():
    """L = 2: layer 0 FP16 with epilogue (1/s_1, b_0/s_1), E4M3 activations, layer 1 E4M3
    weights scaled by s_w = max|W_1| / 448, epilogue (s_w s_1, b_1), FP32 head."""
    rng = np.random.default_rng(5)
    nin, w = 8, 8
    q = rng.integers(0, 2 ** 32, (nin // 2, 3), dtype=np.uint64).astype(np.uint32)
    net = dict(W=[Q.f16(rng.standard_normal((w, nin)) * 0.5), rng.standard_normal((w, w)) * 0.5],
               b=[rng.standard_normal(w) * 0.1, rng.standard_normal(w) * 0.1], wh=rng.standard_normal(w), bh=0.1)
    ep = Q.fp8_epilogue(net, q, 5)
    # the activation range of layer 1's input: min(16 amax, bound)
    zc = N.encode(Q.calib_coords(5), q)
    amax = np.max(np.maximum(zc @ net["W"][0].T + net["b"][0], 0))
    bound = np.max(np.abs(net["W"][0]).sum(1) + np.abs(net["b"][0]))
    s1 = min(16 * amax, bound) / 448.0
    sw = np.max(np.abs(net["W"][1])) / 448.0
    assert ep[0][0] == pytest.approx(1 / s1) and ep[1][0] == pytest.approx(sw * s1)
    z = Q.f16(rng.uniform(-1, 1, (100, nin)))
    a0 = z @ net["W"][0].T
    hq = Q.e4m3(np.maximum((a0 + net["b"][0]) / s1, 0))
    a1 = hq @ Q.e4m3(net["W"][1] / sw).T
    want = np.maximum(sw * s1 * a1 + net["b"][1], 0) @ net["wh"] + net["bh"]
    assert np.allclose(Q.forward(net, z, Q.PREC_FP8, q, 5), want, rtol=1e-6, atol=1e-6)
    # and FP8 is coarse: far from the FP64 forward compared with FP16
    exact, _ = N.forward(net, z)
    assert np.abs(want - exact).max() > 10 * np.abs(Q.forward(net, z, Q.PREC_FP16) - exact).max()


def test_calibration_points_follow_splitmix64():
    from oracle import rng as R
    c = Q.calib_coords(7, n=4)
    for s in range(4):
        z = R.splitmix64(Q.FP8_CALIB_SEED, s)
        assert list(c[s]) == [z & 127, (z >> 21) & 127, (z >> 42) & 127]
