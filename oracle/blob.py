"""Reader/writer of the model blob (the interchange format of nvdb_model_export/import).

Layout, little-endian; every array starts at an 8-byte aligned offset from the
blob start, padding bytes are zero:

  header (128 bytes)
    0   char[8]  magic "NVDBMDL1"      8   uint32 version (1; 2 with a domain decomposition)
    12  uint32   grid_class (0 level set, 1 fog)
    16  float32  background            20  float32 half_width
    24  int32[3] origin                36  int32 log2_extent
    40  int32[2] ffm_size (level 1, level 0)
    48  int32[3] width  (net 0 = level-1 classifier, 1 = level-0 classifier, 2 = voxel regressor)
    60  int32[3] layers (hidden layers per net)
    72  int32    n_patch_sets          76  int32 experts (version 2; reserved 0 in version 1)
    80  int64    n_l2, n_l1, n_leaf, n_active
    112 uint64   subdomain size S, halo h (version 2; reserved 0 in version 1)
  uint32 q1[m1][3], then uint32 q0[m0][3]         (m = ffm_size / 2)
  per net (expert-major: expert k's net j is net 3k + j):
           float32 W_0[w][n], b_0[w], W_1[w][w], b_1[w], ..., w_h[w], b_h
  version 2 only (Section 3.4): int32 dims[3] (+ pad), int32 expert_of[dims product]
           (expert id of each grid subdomain, x-major, -1 = discarded), int32 origin[experts][3]
  int32  l2_origin[n_l2][3]
  uint64 l2_mask[n_l2][512]
  per patch set: int32 precision, int32 reserved,
                 uint32 l1_off[n_l1+1], uint16 l1_idx[l1_off[n_l1]],
                 uint32 l0_off[n_leaf+1], uint16 l0_idx[l0_off[n_leaf]]
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"NVDBMDL1"
HEADER = struct.Struct("<8sIIff3ii2i3i3iii4q2Q")
assert HEADER.size == 128


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


def write(model: dict) -> bytes:
    m = model
    moe = m.get("moe")
    n_exp = 0 if moe is None else len(moe["origins"])
    buf = bytearray(HEADER.pack(
        MAGIC, 1 if moe is None else 2, m["grid_class"], m["background"], m["half_width"], *[int(v) for v in m["origin"]],
        m["log2_extent"], *m["ffm_size"], *m["width"], *m["layers"], len(m["patches"]), n_exp,
        m["n_l2"], m["n_l1"], m["n_leaf"], m["n_active"], 0 if moe is None else moe["size"],
        0 if moe is None else moe["halo"]))
    for q in m["q"]:
        buf += np.ascontiguousarray(q, dtype="<u4").tobytes(); _pad8(buf)
    for k, net in enumerate(m["nets"]):
        for W, b in zip(net["W"], net["b"]):
            buf += np.asarray(W, dtype="<f4").tobytes()
            buf += np.asarray(b, dtype="<f4").tobytes()
        buf += np.asarray(net["wh"], dtype="<f4").tobytes()
        buf += np.asarray([net["bh"]], dtype="<f4").tobytes()
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
    if h[0] != MAGIC or h[1] not in (1, 2):
        raise ValueError("not a model blob")
    version, n_exp = h[1], (h[18] if h[1] == 2 else 1)
    (grid_class, background, half_width) = h[2], h[3], h[4]
    origin = np.array(h[5:8], dtype=np.int64)
    log2e = h[8]
    ffm = list(h[9:11]); width = list(h[11:14]); layers = list(h[14:17])
    n_sets = h[17]
    n_l2, n_l1, n_leaf, n_active = h[19:23]
    o = HEADER.size

    def take(dtype, count):
        nonlocal o
        a = np.frombuffer(data, dtype=dtype, count=count, offset=o).copy()
        o += a.nbytes
        o += (-o) % 8
        return a

    q = [take("<u4", (ffm[0] // 2) * 3).reshape(-1, 3), take("<u4", (ffm[1] // 2) * 3).reshape(-1, 3)]
    nets = []
    for kk in range(3 * n_exp):
        k = kk % 3
        n_in = ffm[0] if k == 0 else ffm[1]
        shapes = _net_shapes(n_in, width[k], layers[k])
        cnt = sum(int(np.prod(s)) for s in shapes)
        flat = take("<f4", cnt).astype(np.float64)
        net = dict(W=[], b=[])
        p = 0
        for i, s in enumerate(shapes):
            sz = int(np.prod(s))
            a = flat[p:p + sz].reshape(s); p += sz
            if i < 2 * layers[k]:
                (net["W"] if i % 2 == 0 else net["b"]).append(a)
            elif i == 2 * layers[k]:
                net["wh"] = a
            else:
                net["bh"] = float(a[0])
        nets.append(net)
    moe = None
    if version == 2:
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
                n_active=n_active, patches=patches, moe=moe)
