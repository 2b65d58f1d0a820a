"""Shared helpers of the GPU parity tests (no GPU work at import time)."""
import numpy as np

from oracle import codec
from oracle import nets as N


def oracle_forward_scale(model: dict, net: int, ijk: np.ndarray):
    """Oracle output and the dot-product error scale sum_i |w_h,i h_i| + |b_h| of the head."""
    z = N.encode(codec.level_coords(model, net, ijk), codec.level_q(model, net))
    y, (hs, _) = N.forward(model["nets"][net], z)
    scale = np.abs(hs[-1] * model["nets"][net]["wh"][None]).sum(1) + abs(model["nets"][net]["bh"])
    return y, scale


def rel_err(gpu: np.ndarray, ref: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """|gpu - ref| / max(|ref|, scale): relative error normalised by the head's dot-product scale."""
    return np.abs(np.asarray(gpu, np.float64) - ref) / np.maximum(np.abs(ref), np.maximum(scale, 1e-30))


def randomise_biases(model: dict, seed: int, s: float = 0.1):
    """Give every bias a random FP32-representable value so parity tests exercise them."""
    r = np.random.default_rng(seed)
    for net in model["nets"]:
        net["b"] = [(r.standard_normal(b.shape) * s).astype(np.float32).astype(np.float64) for b in net["b"]]
        net["bh"] = float(np.float32(r.standard_normal() * s))
    return model


# Decoded-value bars of the tensor-core precisions, as a fraction of the band half-width
# (absolute for fog densities).  FP16 (11 significant bits) and compensated BF16 (hi + lo
# pairs, ~16 bits) meet the 2e-2 target.  Plain BF16 (8 significant bits per activation)
# does not: its measured error on the test and bench models is 2.3e-2 to 2.5e-2 of the
# half-width, so it is held to 5e-2 and its error is reported next to the others.  FP8
# (E4M3 hidden layers, 4 significant bits) is coarser again: held to the half-width.
TC_BARS = {1: 5e-2, 2: 1.0, 3: 2e-2, 4: 2e-2}


def tc_bar(prec: int) -> float:
    return TC_BARS[prec]


def round_bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    u = np.asarray(a, np.float32).copy().view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_weight_sensitivity(net: dict, z: np.ndarray, gy_of) -> np.ndarray:
    """FP64 gradient of the network with its weights and biases rounded to BF16 (the head
    kept): how far one BF16 rounding moves the gradient.  gy_of(y) -> dL/dy."""
    pb = dict(W=[round_bf16(W) for W in net["W"]], b=[round_bf16(b) for b in net["b"]], wh=net["wh"], bh=net["bh"])
    y, cache = N.forward(pb, z)
    return N.flatten(N.backward(pb, cache, gy_of(y)))
