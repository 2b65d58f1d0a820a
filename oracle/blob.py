"""Reader/writer of the model blob (the interchange format of nvdb_model_export/import).

Layout, little-endian; every array starts at an 8-byte aligned offset from the
blob start, padding bytes are zero:

  header (128 bytes)
    0   char[8]  magic "NVDBMDL1"      8   uint32 version (1; 2 with a domain decomposition;
                                           3 with the extension below)
    12  uint32   grid_class (0 level set, 1 fog)
    16  float32  background            20  float32 half_width
    24  int32[3] origin                36  int32 log2_extent
    40  int32[2] ffm_size (level 1, level 0)
    48  int32[3] width  (net 0 = level-1 classifier, 1 = level-0 classifier, 2 = voxel regressor)
    60  int32[3] layers (hidden layers per net)
    72  int32    n_patch_sets          76  int32 experts (version 2; reserved 0 in version 1)
    80  int64    n_l2, n_l1, n_leaf, n_active
    112 uint64   subdomain size S, halo h (versions 2, 3; reserved 0 in version 1)
  version 3 only, extension (32 bytes):
    128 int32 flags (bit 0: ternary level-1 classifier with a tile value regressor)
    132 int32 activation (0 ReLU, 1 sin)   136 float32 omega (sin frequency)
    140 int32 tile regressor width         144 int32 tile regressor hidden layers
    148 int32 reserved 0                   152 int64 active tiles of the source grid
  uint32 q1[m1][3], then uint32 q0[m0][3]         (m = ffm_size / 2)
  per net (expert-major: expert k's net j is net 3k + j; with tiles, net 3 is the tile
  value regressor, on the level-1 encoding):
           float32 W_0[w][n], b_0[w], W_1[w][w], b_1[w], ..., W_h[c][w], b_h[c]
           (c = 3 outputs for the ternary classifier, else 1)
  with experts (version 2, or version 3 with experts > 0; Section 3.4):
           int32 dims[3] (+ pad), int32 expert_of[dims product]
           (expert id of each grid subdomain, x-major, -1 = discarded), int32 origin[experts][3]
  int32  l2_origin[n_l2][3]
  uint64 l2_mask[n_l2][512]
  per patch set: int32 precision, int32 reserved,
                 uint32 l1_off[n_l1+1], uint16 l1_idx[l1_off[n_l1]]  (ternary: slot | class << 12),
                 uint32 l0_off[n_leaf+1], uint16 l0_idx[l0_off[n_leaf]]
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"NVDBMDL1"
HEADER = struct.Struct("<8sIIff3ii2i3i3iii4q2Q")
EXT = struct.Struct("<iifiiiq")
assert HEADER.size == 128 and EXT.size == 32


def _pad8(buf: bytearray):
    buf.extend(b"\0" * ((-len(buf)) % 8))


def _net_shapes(n_in: int, width: int, layers: int):
    shapes = []
    fan = n_in
    for _ in range(layers):
        shapes += [(width, fan), (width,)]
        fan = width
    shapes += [(width,), (1,)]
    return shapes


def _net_shapes_out(n_in: int, width: int, layers: int, n_out: int):
    s = _net_shapes(n_in, width, layers)
    return s if n_out == 1 else s[:-2] + [(n_out, width), (n_out,)]


def write(model: dict) -> bytes:
    m = model
    moe = m.get("moe")
    n_exp = 0 if moe is None else len(moe["origins"])
    ext = m.get("ternary", False) or m.get("act", 0) != 0
    buf = bytearray(HEADER.pack(
        MAGIC, 3 if ext else (1 if moe is None else 2), m["grid_class"], m["background"], m["half_width"], *[int(v) for v in m["origin"]],
        m["log2_extent"], *m["ffm_size"], *m["width"], *m["layers"], len(m["patches"]), n_exp,
        m["n_l2"], m["n_l1"], m["n_leaf"], m["n_active"], 0 if moe is None else moe["size"],
        0 if moe is None else moe["halo"]))
    if ext:
        tw, tl = m.get("tile_shape", (0, 0)) if m.get("ternary") else (0, 0)
        buf += EXT.pack(1 if m.get("ternary") else 0, m.get("act", 0), m.get("omega", 1.0), tw, tl, 0,
                        m.get("n_tiles", 0))
    for q in m["q"]:
        buf += np.ascontiguousarray(q, dtype="<u4").tobytes(); _pad8(buf)
    for k, net in enumerate(m["nets"]):
        for W, b in zip(net["W"], net["b"]):
            buf += np.asarray(W, dtype="<f4").tobytes()
            buf += np.asarray(b, dtype="<f4").tobytes()
        buf += np.asarray(net["wh"], dtype="<f4").tobytes()
        buf += np.asarray(net["bh"], dtype="<f4").reshape(-1).tobytes()
        _pad8(buf)
    if moe is not None:
        buf += np.asarray(moe["dims"], dtype="<i4").tobytes(); _pad8(buf)
        buf += np.asarray(moe["expert_of"], dtype="<i4").tobytes(); _pad8(buf)
        buf += np.asarray(moe["origins"], dtype="<i4").tobytes(); _pad8(buf)
    buf += np.asarray(m["l2_origin"], dtype="<i4").tobytes(); _pad8(buf)
    buf += np.asarray(m["l2_mask"], dtype="<u8").tobytes(); _pad8(buf)
    for prec in sorted(m["patches"]):
        p = m["patches"][prec]
        buf += struct.pack("<ii", prec, 0)
        buf += np.asarray(p["l1_off"], dtype="<u4").tobytes(); _pad8(buf)
        buf += np.asarray(p["l1_idx"], dtype="<u2").tobytes(); _pad8(buf)
        buf += np.asarray(p["l0_off"], dtype="<u4").tobytes(); _pad8(buf)
        buf += np.asarray(p["l0_idx"], dtype="<u2").tobytes(); _pad8(buf)
    return bytes(buf)


def read(data: bytes) -> dict:
    h = HEADER.unpack_from(data, 0)
    if h[0] != MAGIC or h[1] not in (1, 2, 3):
        raise ValueError("not a model blob")
    version = h[1]
    has_moe = version == 2 or (version == 3 and h[18] > 0)
    n_exp = h[18] if has_moe else 1
    (grid_class, background, half_width) = h[2], h[3], h[4]
    origin = np.array(h[5:8], dtype=np.int64)
    log2e = h[8]
    ffm = list(h[9:11]); width = list(h[11:14]); layers = list(h[14:17])
    n_sets = h[17]
    n_l2, n_l1, n_leaf, n_active = h[19:23]
    o = HEADER.size
    ternary, act, omega, tile_shape, n_tiles = False, 0, 1.0, (0, 0), 0
    if version == 3:
        flags, act, omega, tw, tl, _r, n_tiles = EXT.unpack_from(data, o)
        o += EXT.size
        ternary, tile_shape = bool(flags & 1), (tw, tl)

    def take(dtype, count):
        nonlocal o
        a = np.frombuffer(data, dtype=dtype, count=count, offset=o).copy()
        o += a.nbytes
        o += (-o) % 8
        return a

    q = [take("<u4", (ffm[0] // 2) * 3).reshape(-1, 3), take("<u4", (ffm[1] // 2) * 3).reshape(-1, 3)]
    nets = []
    for kk in range(3 * n_exp + (1 if ternary else 0)):
        k = kk % 3 if kk < 3 * n_exp else 3
        n_in = ffm[0] if k in (0, 3) else ffm[1]
        w_k, l_k = (width[k], layers[k]) if k < 3 else tile_shape
        shapes = _net_shapes_out(n_in, w_k, l_k, 3 if (ternary and k == 0) else 1)
        cnt = sum(int(np.prod(s)) for s in shapes)
        flat = take("<f4", cnt).astype(np.float64)
        net = dict(W=[], b=[], act=act, omega=float(np.float32(omega)))
        p = 0
        for i, s in enumerate(shapes):
            sz = int(np.prod(s))
            a = flat[p:p + sz].reshape(s); p += sz
            if i < 2 * l_k:
                (net["W"] if i % 2 == 0 else net["b"]).append(a)
            elif i == 2 * l_k:
                net["wh"] = a
            else:
                net["bh"] = float(a[0]) if s == (1,) else a
        nets.append(net)
    moe = None
    if has_moe:
        dims = tuple(int(v) for v in take("<i4", 3))
        expert_of = take("<i4", dims[0] * dims[1] * dims[2]).astype(np.int32)
        origins = take("<i4", n_exp * 3).reshape(-1, 3).astype(np.int64)
        moe = dict(size=int(h[23]), halo=int(h[24]), dims=dims, expert_of=expert_of, origins=origins)
    l2_origin = take("<i4", n_l2 * 3).reshape(-1, 3).astype(np.int64)
    l2_mask = take("<u8", n_l2 * 512).reshape(-1, 512)
    patches = {}
    for _ in range(n_sets):
        prec, _r = struct.unpack_from("<ii", data, o); o += 8
        l1_off = take("<u4", n_l1 + 1)
        l1_idx = take("<u2", int(l1_off[-1]))
        l0_off = take("<u4", n_leaf + 1)
        l0_idx = take("<u2", int(l0_off[-1]))
        patches[prec] = dict(l1_off=l1_off, l1_idx=l1_idx, l0_off=l0_off, l0_idx=l0_idx)
    return dict(grid_class=grid_class, background=background, half_width=half_width, origin=origin,
                log2_extent=log2e, ffm_size=ffm, width=width, layers=layers, q=q, nets=nets,
                l2_origin=l2_origin, l2_mask=l2_mask, n_l2=n_l2, n_l1=n_l1, n_leaf=n_leaf,
                n_active=n_active, patches=patches, moe=moe, ternary=ternary, act=act,
                omega=float(np.float32(omega)), tile_shape=tile_shape, n_tiles=n_tiles)
