"""Counter-based generators and the parameter initialisation drawn from them.

* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): draw i of a stream with seed s is
  mix64(s + (i+1) * 0x9E3779B97F4A7C15), i.e. the (i+1)-th output of the
  sequential generator started at state s.
* Philox4x32-10 (Salmon et al., "Parallel random numbers: as easy as 1, 2,
  3", SC 2011): 10 rounds of the 4x32 multiply/xor round with Weyl key
  schedule.

Initialisation (the paper uses standard practice without stating it; these
are the readings):
* Xavier-uniform weights W ~ U(-a, a), a = sqrt(6 / (fan_in + fan_out)),
  drawn in FP64 and rounded to FP32; biases 0.
* Fourier matrix B ~ N(0, sigma^2) by Box-Muller (Tancik et al. 2020, the FFM
  the paper adopts in Section 3.2.2), stored as fixed-point phase increments
  q = rint(2^32 * B / E) mod 2^32, E the level's power-of-two extent.
"""
from __future__ import annotations

import math

import numpy as np

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
NET_STREAM = 0x632BE59BD9B4E019   # stream offset of network k: seed + NET_STREAM*(k+1)
FFM_STREAM = 0x8CB92BA72F3D8DD7   # stream offset of encoding level l: seed + FFM_STREAM*(l+1)


def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def splitmix64(seed: int, i: int) -> int:
    """Draw i (0-based) of the SplitMix64 stream started at state ``seed``."""
    return _mix64((seed + (i + 1) * GOLDEN) & M64)


def uniform01(seed: int, i: int) -> float:
    """Draw i as a double in [0, 1): top 53 bits times 2^-53."""
    return (splitmix64(seed, i) >> 11) * (1.0 / 9007199254740992.0)


# ----------------------------------------------------------------- Philox4x32-10

PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds on uint32 arrays.

    ctr: array [..., 4] (uint32), key: array [..., 2] (uint32).  Returns [..., 4] uint32.
    One round: (c0,c1,c2,c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0));
    the key is bumped by the Weyl constants before every round but the first.
    """
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64)
    k1 = np.asarray(key[..., 1], dtype=np.uint64)
    m32 = np.uint64(0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(PHILOX_W0)) & m32
            k1 = (k1 + np.uint64(PHILOX_W1)) & m32
        p0 = np.uint64(PHILOX_M0) * c[0]
        p1 = np.uint64(PHILOX_M1) * c[2]
        c = [((p1 >> np.uint64(32)) ^ c[1] ^ k0) & m32, p1 & m32,
             ((p0 >> np.uint64(32)) ^ c[3] ^ k1) & m32, p0 & m32]
    return np.stack(c, -1).astype(np.uint32)


def sample_indices(seed: int, net: int, step: int, batch: int, population: int) -> np.ndarray:
    """Training-sample indices of one step (Section 3.2.1: uniform over the population).

    Sample s uses word (s mod 4) of Philox4x32-10 with counter (s div 4, step, net, 0)
    and key (seed low 32 bits, seed high 32 bits); index = floor(u32 * population / 2^32).
    """
    if not (0 < population < (1 << 32)):
        raise ValueError("population must be in [1, 2^32)")
    nblk = (batch + 3) // 4
    ctr = np.zeros((nblk, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(nblk)
    ctr[:, 1] = step
    ctr[:, 2] = net
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    out = philox4x32_10(ctr, np.broadcast_to(key, (nblk, 2))).reshape(-1)[:batch]
    return ((out.astype(np.uint64) * np.uint64(population)) >> np.uint64(32)).astype(np.int64)


def subset_indices(seed: int, net: int, step: int, batch: int, interval: int, population: int) -> np.ndarray:
    """Training-sample indices with subset resampling (Appendix E): every `interval` steps a
    subset of interval * batch candidates is drawn, and each step draws its batch from it.
    Sample s of step t takes the position p = sample_indices(...)[s] in the subset of size
    interval * batch, then subset element p of interval r = (t - 1) div interval: word (p mod 4)
    of Philox4x32-10 with counter (p div 4, r, net, 1), scaled to the population."""
    if not (0 < population < (1 << 32)):
        raise ValueError("population must be in [1, 2^32)")
    pos = sample_indices(seed, net, step, batch, interval * batch).astype(np.uint64)
    ctr = np.zeros((len(pos), 4), dtype=np.uint64)
    ctr[:, 0] = pos >> np.uint64(2)
    ctr[:, 1] = (step - 1) // interval
    ctr[:, 2] = net
    ctr[:, 3] = 1
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    words = philox4x32_10(ctr, np.broadcast_to(key, (len(pos), 2)))
    u = words[np.arange(len(pos)), (pos & np.uint64(3)).astype(np.int64)].astype(np.uint64)
    return ((u * np.uint64(population)) >> np.uint64(32)).astype(np.int64)


# ----------------------------------------------------------------- initialisation

def xavier_net(seed: int, net: int, n_in: int, width: int, layers: int, n_out: int = 1) -> dict:
    """Initial parameters of one MLP: `layers` hidden layers of `width`, then a head of
    n_out outputs.

    Draw order on stream seed + NET_STREAM*(net+1): W_0 row-major [width][n_in], then
    W_1..W_{layers-1} [width][width], then the head W_h row-major [n_out][width] (a vector
    [width] for one output), bound sqrt(6 / (width + n_out)).  Biases are zero.
    """
    s = (seed + NET_STREAM * (net + 1)) & M64
    i = 0
    Ws, bs = [], []
    fan = [n_in] + [width] * layers
    for l in range(layers):
        a = math.sqrt(6.0 / (fan[l] + width))
        W = np.empty((width, fan[l]), dtype=np.float64)
        for o in range(width):
            for c in range(fan[l]):
                W[o, c] = (2.0 * uniform01(s, i) - 1.0) * a
                i += 1
        Ws.append(W.astype(np.float32).astype(np.float64))
        bs.append(np.zeros(width))
    a = math.sqrt(6.0 / (width + n_out))
    wh = np.empty((n_out, width))
    for o in range(n_out):
        for c in range(width):
            wh[o, c] = (2.0 * uniform01(s, i) - 1.0) * a
            i += 1
    wh = wh.astype(np.float32).astype(np.float64)
    if n_out == 1:
        return dict(W=Ws, b=bs, wh=wh[0], bh=0.0)
    return dict(W=Ws, b=bs, wh=wh, bh=np.zeros(n_out))


def ffm_increments(seed: int, level: int, m: int, sigma: float, extent: int) -> np.ndarray:
    """Fixed-point Fourier matrix of one level: q[f, d] = rint(2^32 * B[f, d] / extent) mod 2^32.

    B[f, d] = sigma * sqrt(-2 ln(1 - u1)) * cos(2 pi u2) with u1, u2 draws 2i, 2i+1 (i = 3f + d)
    of stream seed + FFM_STREAM*(level+1).
    """
    s = (seed + FFM_STREAM * (level + 1)) & M64
    q = np.zeros((m, 3), dtype=np.uint32)
    for f in range(m):
        for d in range(3):
            i = 3 * f + d
            u1, u2 = uniform01(s, 2 * i), uniform01(s, 2 * i + 1)
            z = math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)
            t = math.ldexp(sigma * z, 32) / extent
            q[f, d] = int(np.rint(t)) % (1 << 32)
    return q
