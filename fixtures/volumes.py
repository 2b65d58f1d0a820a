"""Seeded generators of sparse volumes (narrow-band level sets and fog).

The volumes stand in for the paper's datasets (Stanford models, Disney Cloud,
EmberGen, ...), which are not available: they have the same structure -- a
narrow band of half-width ``w`` voxels around a surface (level sets, Section
3.2.1: active voxels lie in the band [-3dx, 3dx]) or a bounded fog with a
non-trivial boundary -- at the sizes of the benchmark workloads.

All generators are deterministic functions of their arguments.  They run on
any torch device; every per-voxel formula is written as separate elementwise
torch ops (no fused multiply-add), so the CPU and CUDA results agree.

Outputs: ``ijk`` int32 [n, 3] (non-negative voxel coordinates) and ``val``
float32 [n] (signed distance in voxel units, or density).  The order of the
voxels is unspecified; the tree build sorts them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

F64 = torch.float64


def _half_diag(s: int) -> float:
    """Largest distance from the centre of an s^3 block of voxel centres to any of them."""
    return (s - 1) / 2.0 * math.sqrt(3.0)


@dataclass
class Primitive:
    kind: str                   # "sphere" or "torus" (torus axis = local y)
    centre: tuple
    radius: float               # sphere radius, or torus tube radius r
    major: float = 0.0          # torus ring radius R
    rot: np.ndarray = field(default_factory=lambda: np.eye(3))  # columns = local axes in world


def _shoemake_rotation(u1: float, u2: float, u3: float) -> np.ndarray:
    """Uniformly random rotation from three U[0,1) numbers (Shoemake, Graphics Gems III)."""
    a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
    x, y = a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2)
    z, w = b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def random_primitives(grid: int, n_spheres: int, n_tori: int, seed: int,
                      sphere_r=(20.0, 120.0), torus_R=(40.0, 160.0),
                      torus_r=(8.0, 30.0)) -> list:
    """Seeded spheres and tori with centres uniform in [0, grid)^3 and uniform random orientation."""
    rng = np.random.Generator(np.random.PCG64(seed))
    prims = []
    for _ in range(n_spheres):
        c = tuple(float(v) for v in rng.uniform(0.0, grid, 3))
        prims.append(Primitive("sphere", c, float(rng.uniform(*sphere_r))))
    for _ in range(n_tori):
        c = tuple(float(v) for v in rng.uniform(0.0, grid, 3))
        R = float(rng.uniform(*torus_R))
        r = float(rng.uniform(*torus_r))
        u = rng.uniform(0.0, 1.0, 3)
        prims.append(Primitive("torus", c, r, R, _shoemake_rotation(*u)))
    return prims


class _PrimTable:
    """Primitive parameters as device tensors, indexed per (point, primitive) pair."""

    def __init__(self, prims, device):
        self.n = len(prims)
        self.is_torus = torch.tensor([p.kind == "torus" for p in prims], device=device)
        self.c = torch.tensor([p.centre for p in prims], dtype=F64, device=device)
        self.r = torch.tensor([p.radius for p in prims], dtype=F64, device=device)
        self.R = torch.tensor([p.major for p in prims], dtype=F64, device=device)
        self.rot = torch.tensor(np.stack([p.rot for p in prims]), dtype=F64, device=device)

    def sdf(self, p: torch.Tensor, j: torch.Tensor) -> torch.Tensor:
        """Exact signed distance of primitive j[k] at point p[k] (float64 [K,3] -> [K])."""
        dx = p[:, 0] - self.c[j, 0]
        dy = p[:, 1] - self.c[j, 1]
        dz = p[:, 2] - self.c[j, 2]
        sph = torch.sqrt(dx * dx + dy * dy + dz * dz) - self.r[j]
        m = self.rot[j]
        lx = dx * m[:, 0, 0] + dy * m[:, 1, 0] + dz * m[:, 2, 0]
        ly = dx * m[:, 0, 1] + dy * m[:, 1, 1] + dz * m[:, 2, 1]
        lz = dx * m[:, 0, 2] + dy * m[:, 1, 2] + dz * m[:, 2, 2]
        qx = torch.sqrt(lx * lx + lz * lz) - self.R[j]
        tor = torch.sqrt(qx * qx + ly * ly) - self.r[j]
        return torch.where(self.is_torus[j], tor, sph)


def _cube_offsets(f: int, device) -> torch.Tensor:
    a = torch.arange(f, device=device)
    g = torch.stack(torch.meshgrid(a, a, a, indexing="ij"), -1).reshape(-1, 3)
    return g.to(torch.int64)


def primitives_union(prims, grid: int, half_width: float = 3.0, device="cpu",
                     chunk: int = 1 << 22):
    """Narrow band of the union (min) of exact primitive SDFs, clipped to [0, grid)^3.

    A voxel is active iff |d| < half_width (strict); its value is d.  The band
    is found by refining (block, primitive) pairs: every exact SDF is
    1-Lipschitz, so a primitive whose distance at a block centre exceeds
    ``half_width + half_diagonal`` cannot change the union's band inside that
    block and is dropped for it.
    """
    dev = torch.device(device)
    tab = _PrimTable(prims, dev)
    w = float(half_width)
    sizes = [s for s in (512, 64, 8) if s <= grid and grid % s == 0]
    if not sizes or sizes[-1] != 8:
        raise ValueError("grid must be a multiple of 8")
    top = sizes[0]
    nb = grid // top
    org = _cube_offsets(nb, dev) * top
    # all (top block, primitive) pairs
    blk = org.repeat_interleave(tab.n, 0)
    pj = torch.arange(tab.n, device=dev).repeat(org.shape[0])
    s = top
    levels = sizes[1:] + [1]
    for child in levels:
        # keep pairs whose primitive can reach the band inside the block
        keep_parts = []
        for a in range(0, blk.shape[0], chunk):
            b = blk[a:a + chunk]
            cen = b.to(F64) + (s - 1) / 2.0
            d = tab.sdf(cen, pj[a:a + chunk])
            keep_parts.append(d <= w + _half_diag(s))
        keep = torch.cat(keep_parts) if keep_parts else torch.zeros(0, dtype=torch.bool, device=dev)
        blk, pj = blk[keep], pj[keep]
        if child == 1:
            break
        f = s // child
        off = _cube_offsets(f, dev) * child
        nparent = blk.shape[0]
        blk = (blk[:, None, :] + off[None, :, :]).reshape(-1, 3)
        pj = pj.repeat_interleave(off.shape[0])
        del nparent
        s = child
    # voxel level: pairs (8^3 block, primitive) -> per-voxel min over the block's primitives,
    # one chunk of blocks (in key order) at a time so that memory stays bounded
    assert s == 8
    key = (blk[:, 0] * grid + blk[:, 1]) * grid + blk[:, 2]
    key, order = torch.sort(key)
    pj = pj[order]
    del blk, order
    ublk, counts = torch.unique_consecutive(key, return_counts=True)
    del key
    ends = torch.cumsum(counts, 0)
    ends_h = ends.cpu()
    off8 = _cube_offsets(8, dev)
    bstep = max(1, chunk // 512)
    outs_ijk, outs_val = [], []
    for a in range(0, ublk.shape[0], bstep):
        b_hi = min(a + bstep, ublk.shape[0])
        p_lo = int(ends_h[a - 1]) if a > 0 else 0
        p_hi = int(ends_h[b_hi - 1])
        ub = ublk[a:b_hi]
        borg = torch.stack([ub // (grid * grid), (ub // grid) % grid, ub % grid], 1)
        dmin = torch.full((b_hi - a, 512), float("inf"), dtype=F64, device=dev)
        # block of each pair, relative to the chunk
        rel = torch.repeat_interleave(torch.arange(b_hi - a, device=dev), counts[a:b_hi])
        for q in range(p_lo, p_hi, bstep):
            r = rel[q - p_lo:min(q + bstep, p_hi) - p_lo]
            vox = (borg[r][:, None, :] + off8[None]).reshape(-1, 3)
            jj = pj[q:q + r.shape[0]].repeat_interleave(512)
            d = tab.sdf(vox.to(F64), jj).reshape(-1, 512)
            dmin.scatter_reduce_(0, r[:, None].expand(-1, 512), d, reduce="amin")
        vox = (borg[:, None, :] + off8[None]).reshape(-1, 3)
        d = dmin.reshape(-1)
        inside = ((vox >= 0) & (vox < grid)).all(1)
        act = inside & (d.abs() < w)
        outs_ijk.append(vox[act].to(torch.int32))
        outs_val.append(d[act].to(torch.float32))
    if not outs_ijk:
        return torch.zeros((0, 3), dtype=torch.int32, device=dev), torch.zeros(0, dtype=torch.float32, device=dev)
    return torch.cat(outs_ijk), torch.cat(outs_val)


def sphere_band(grid=128, centre=(64.0, 64.0, 64.0), radius=40.0, half_width=3.0, device="cpu"):
    """Narrow-band SDF of one sphere (voxel centres at integer coordinates)."""
    return primitives_union([Primitive("sphere", tuple(map(float, centre)), float(radius))],
                            grid, half_width, device)


# --------------------------------------------------------------------------- fog

def _mul32(x: torch.Tensor, c: int) -> torch.Tensor:
    """Low 32 bits of x*c for 0 <= x < 2^32, computed without int64 overflow."""
    lo = x * (c & 0xFFFF)
    hi = ((x * (c >> 16)) & 0xFFFF) << 16
    return (lo + hi) & 0xFFFFFFFF


def _lowbias32(x: torch.Tensor) -> torch.Tensor:
    """32-bit integer hash 'lowbias32' (C. Wellons, hash-prospector)."""
    x = x ^ (x >> 16)
    x = _mul32(x, 0x7FEB352D)
    x = x ^ (x >> 15)
    x = _mul32(x, 0x846CA68B)
    return x ^ (x >> 16)


def _lattice_value(seed: int, octave: int, lx, ly, lz) -> torch.Tensor:
    """Value in [-1, 1) attached to an integer lattice point of one octave."""
    h = _lowbias32(torch.full_like(lx, (seed ^ ((octave * 0x9E3779B9) & 0xFFFFFFFF)) & 0xFFFFFFFF))
    h = _lowbias32((lx & 0xFFFFFFFF) ^ h)
    h = _lowbias32((ly & 0xFFFFFFFF) ^ h)
    h = _lowbias32((lz & 0xFFFFFFFF) ^ h)
    return h.to(F64) * (2.0 / 4294967296.0) - 1.0


def _value_noise(p: torch.Tensor, period: float, seed: int, octave: int) -> torch.Tensor:
    x = p / period
    cell = torch.floor(x)
    t = x - cell
    s = t * t * (3.0 - 2.0 * t)
    ci = cell.to(torch.int64)
    out = torch.zeros(p.shape[0], dtype=F64, device=p.device)
    for a in (0, 1):
        wa = s[:, 0] if a else 1.0 - s[:, 0]
        for b in (0, 1):
            wb = s[:, 1] if b else 1.0 - s[:, 1]
            for c in (0, 1):
                wc = s[:, 2] if c else 1.0 - s[:, 2]
                v = _lattice_value(seed, octave, ci[:, 0] + a, ci[:, 1] + b, ci[:, 2] + c)
                out = out + (wa * wb) * wc * v
    return out


def fbm_noise(p: torch.Tensor, octaves=6, lacunarity=2.0, gain=0.5, seed=3, base_period=64.0) -> torch.Tensor:
    """The fBm of fbm_fog remapped to [0, 1], at arbitrary (float) points p [N, 3]: a continuous
    function (smoothstep-blended lattice values), the ground truth of the sampling-error study."""
    p = p.to(F64)
    norm = sum(gain ** o for o in range(octaves))
    acc = torch.zeros(p.shape[0], dtype=F64, device=p.device)
    for o in range(octaves):
        acc = acc + (gain ** o) * _value_noise(p, base_period / (lacunarity ** o), seed, o)
    return (acc / norm + 1.0) * 0.5


def fbm_fog(grid=512, octaves=6, lacunarity=2.0, gain=0.5, seed=3, base_period=64.0,
            axes=(200.0, 150.0, 120.0), centre=None, threshold=0.05, device="cpu",
            chunk: int = 1 << 22):
    """fBm value-noise density remapped to [0,1], times an ellipsoid falloff, zeroed below threshold.

    density(p) = (fbm(p) + 1)/2 * clamp(1 - |(p - c)/a|^2, 0, 1), active iff >= threshold,
    with fbm = sum_o gain^o noise(p * lacunarity^o / base_period) / sum_o gain^o.
    """
    dev = torch.device(device)
    c = torch.tensor(centre if centre is not None else (grid / 2.0,) * 3, dtype=F64, device=dev)
    a = torch.tensor(axes, dtype=F64, device=dev)
    lo = torch.clamp(torch.floor(c - a), 0, grid - 1).to(torch.int64)
    hi = torch.clamp(torch.ceil(c + a), 0, grid - 1).to(torch.int64)
    ext = (hi - lo + 1).tolist()
    total = ext[0] * ext[1] * ext[2]
    norm = sum(gain ** o for o in range(octaves))
    outs_ijk, outs_val = [], []
    for s0 in range(0, total, chunk):
        lin = torch.arange(s0, min(total, s0 + chunk), device=dev)
        z = lin % ext[2]
        y = (lin // ext[2]) % ext[1]
        x = lin // (ext[1] * ext[2])
        ijk = torch.stack([x, y, z], 1) + lo
        p = ijk.to(F64)
        q = (p - c) / a
        fall = torch.clamp(1.0 - (q[:, 0] * q[:, 0] + q[:, 1] * q[:, 1] + q[:, 2] * q[:, 2]), 0.0, 1.0)
        sel = fall >= threshold
        ijk, p, fall = ijk[sel], p[sel], fall[sel]
        acc = torch.zeros(p.shape[0], dtype=F64, device=dev)
        for o in range(octaves):
            acc = acc + (gain ** o) * _value_noise(p, base_period / (lacunarity ** o), seed, o)
        dens = (acc / norm + 1.0) * 0.5 * fall
        keep = dens >= threshold
        outs_ijk.append(ijk[keep].to(torch.int32))
        outs_val.append(dens[keep].to(torch.float32))
    return torch.cat(outs_ijk), torch.cat(outs_val)


# --------------------------------------------------------------------------- water

def tiled_fog(nx: int = 32, ny: int = 24, nz: int = 24, const: float = 0.5):
    """A fog block [0, nx) x [0, ny) x [0, nz) whose x < nx/2 half holds the constant density
    `const` (its full leaves become active tiles under tile pruning), the rest a gradient;
    the full leaf at x >= 24, y, z < 8 spans 0.0077 (a tile only with tolerance >= that), and
    two voxels at x = 40, 41 form a partial leaf.  Returns (ijk int64 [n, 3], val float32 [n])."""
    a = [np.arange(nx), np.arange(ny), np.arange(nz)]
    g = np.stack(np.meshgrid(*a, indexing="ij"), -1).reshape(-1, 3)
    v = np.where(g[:, 0] < nx // 2, const, 0.2 + 0.01 * g[:, 1] + 0.001 * g[:, 2])
    near = (g[:, 0] >= 24) & (g[:, 0] < 32) & (g[:, 1] < 8) & (g[:, 2] < 8)
    v = np.where(near, 0.3 + 0.001 * (g[:, 1] + g[:, 2]) / 2.0, v)
    extra = np.array([[nx + 8, 0, 0], [nx + 9, 3, 2]])
    g = np.concatenate([g, extra])
    v = np.concatenate([v, [const, const]]).astype(np.float32)
    return g.astype(np.int64), v


def water_waves(seed=4, n_waves=8, amp=(2.0, 12.0), wavelength=(32.0, 400.0), speed=(0.5, 2.0)):
    """Seeded sine-wave parameters: amplitude, wavelength, direction angle, phase, speed (voxels/frame)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.uniform(*amp, n_waves)
    lam = rng.uniform(*wavelength, n_waves)
    th = rng.uniform(0.0, 2 * math.pi, n_waves)
    ph = rng.uniform(0.0, 2 * math.pi, n_waves)
    sp = rng.uniform(*speed, n_waves)
    return dict(A=A, lam=lam, theta=th, phase=ph, speed=sp)


def water_frame(frame: int, nx=2048, ny=256, nz=2048, y0=128.0, half_width=3.0, seed=4,
                device="cpu", chunk_cols: int = 1 << 20):
    """Narrow band of the water surface y = h(x,z,t) = y0 + sum_k A_k sin(2pi(d_k.(x,z) - c_k t)/lam_k + phi_k).

    Signed distance approximated to first order: d = (y - h)/sqrt(1 + |grad h|^2).
    """
    dev = torch.device(device)
    wv = water_waves(seed)
    A = torch.tensor(wv["A"], dtype=F64, device=dev)
    k = torch.tensor(2 * math.pi / wv["lam"], dtype=F64, device=dev)
    dx = torch.tensor(np.cos(wv["theta"]), dtype=F64, device=dev)
    dz = torch.tensor(np.sin(wv["theta"]), dtype=F64, device=dev)
    ph = torch.tensor(wv["phase"] - 2 * math.pi * wv["speed"] * frame / wv["lam"], dtype=F64, device=dev)
    w = float(half_width)
    outs_ijk, outs_val = [], []
    ncol = nx * nz
    for s0 in range(0, ncol, chunk_cols):
        lin = torch.arange(s0, min(ncol, s0 + chunk_cols), device=dev)
        x = (lin // nz).to(F64)
        z = (lin % nz).to(F64)
        arg = (x[:, None] * dx[None] + z[:, None] * dz[None]) * k[None] + ph[None]
        h = y0 + (A[None] * torch.sin(arg)).sum(1)
        c = A[None] * k[None] * torch.cos(arg)
        gx = (c * dx[None]).sum(1)
        gz = (c * dz[None]).sum(1)
        sc = torch.sqrt(1.0 + gx * gx + gz * gz)
        ylo = torch.clamp(torch.floor(h - w * sc), 0, ny - 1).to(torch.int64)
        yhi = torch.clamp(torch.ceil(h + w * sc), 0, ny - 1).to(torch.int64)
        cnt = (yhi - ylo + 1).clamp(min=0)
        col = torch.repeat_interleave(torch.arange(lin.shape[0], device=dev), cnt)
        start = torch.cumsum(cnt, 0) - cnt
        y = ylo[col] + (torch.arange(col.shape[0], device=dev) - start[col])
        d = (y.to(F64) - h[col]) / sc[col]
        keep = d.abs() < w
        col, y, d = col[keep], y[keep], d[keep]
        ijk = torch.stack([(lin[col] // nz), y, (lin[col] % nz)], 1)
        outs_ijk.append(ijk.to(torch.int32))
        outs_val.append(d.to(torch.float32))
    return torch.cat(outs_ijk), torch.cat(outs_val)


# --------------------------------------------------------------------------- queries

def query_points(ijk: torch.Tensor, n: int, seed: int = 5) -> torch.Tensor:
    """n float32 points: an occupied 128^3 node picked uniformly, then a point uniform in its box."""
    node = ijk.to(torch.int64) >> 7                  # on the tensor's device
    key = torch.unique((node[:, 0] << 42) | (node[:, 1] << 21) | node[:, 2]).cpu()   # lexicographic order
    del node
    nodes = torch.stack([key >> 42, (key >> 21) & ((1 << 21) - 1), key & ((1 << 21) - 1)], 1).numpy()
    rng = np.random.Generator(np.random.PCG64(seed))
    pick = rng.integers(0, nodes.shape[0], n)
    u = rng.uniform(0.0, 128.0, (n, 3))
    pts = (nodes[pick] * 128).astype(np.float64) + u
    return torch.from_numpy(pts.astype(np.float32))


# --------------------------------------------------------------------------- named workloads

WORKLOADS = {
    # name: (description, generator kwargs, network/training defaults)
    "sphere128": "sphere r=40 centred in 128^3, half-band 3; 3x32 ReLU nets, FFM 32",
    "union1024": "union of 32 spheres + 32 tori (seed 2) in 1024^3, half-band 3; 4x64 nets, FFM 64",
    "fog512": "6-octave fBm fog x ellipsoid (seed 3) in 512^3; regressor 4x64, classifiers 3x32, FFM 64",
    "water2048": "8 seeded sine waves, 2048x256x2048, half-band 3, 48 frames",
    "union4096": "union of 128 spheres + 128 tori (seed 5) in 4096^3, half-band 3",
    # small variants used by CPU tests
    "sphere32": "sphere r=10 centred in 32^3, half-band 3",
    "union128": "union of 3 spheres + 3 tori (seed 7) in 128^3, half-band 3",
    "fog64": "fBm fog x ellipsoid (seed 3) in 64^3, base period 8",
}


def workload(name: str, device="cpu", frame: int = 0):
    """Generate a named workload -> (ijk int32 [n,3], val float32 [n], meta dict)."""
    if name == "sphere128":
        ijk, v = sphere_band(128, (64.0, 64.0, 64.0), 40.0, 3.0, device)
        return ijk, v, dict(grid_class=0, half_width=3.0, grid=128)
    if name == "sphere32":
        ijk, v = sphere_band(32, (16.0, 16.0, 16.0), 10.0, 3.0, device)
        return ijk, v, dict(grid_class=0, half_width=3.0, grid=32)
    if name == "union1024":
        prims = random_primitives(1024, 32, 32, seed=2)
        ijk, v = primitives_union(prims, 1024, 3.0, device)
        return ijk, v, dict(grid_class=0, half_width=3.0, grid=1024)
    if name == "union128":
        prims = random_primitives(128, 3, 3, seed=7, sphere_r=(6.0, 24.0), torus_R=(10.0, 30.0),
                                  torus_r=(3.0, 8.0))
        ijk, v = primitives_union(prims, 128, 3.0, device)
        return ijk, v, dict(grid_class=0, half_width=3.0, grid=128)
    if name == "union4096":
        prims = random_primitives(4096, 128, 128, seed=5, sphere_r=(80.0, 480.0),
                                  torus_R=(160.0, 640.0), torus_r=(32.0, 120.0))
        ijk, v = primitives_union(prims, 4096, 3.0, device)
        return ijk, v, dict(grid_class=0, half_width=3.0, grid=4096)
    if name == "fog512":
        ijk, v = fbm_fog(512, device=device)
        return ijk, v, dict(grid_class=1, half_width=0.0, grid=512)
    if name == "fog64":
        ijk, v = fbm_fog(64, base_period=8.0, axes=(25.0, 19.0, 15.0), device=device)
        return ijk, v, dict(grid_class=1, half_width=0.0, grid=64)
    if name == "water2048":
        ijk, v = water_frame(frame, device=device)
        return ijk, v, dict(grid_class=0, half_width=3.0, grid=2048)
    raise KeyError(name)
