"""The tensor-core kernel variants compute the same bits.

Variant 0 (the default kernel, in its lattice-only and list-only instantiations), 1 (256
threads per tile, split epilogue) and 2 (origins staged by bulk copies) are chosen per
process (NVDB_TC_VARIANT) or by the decode-plan autotuner; whichever runs, the decoded
topology and values, the network outputs at listed coordinates and the point queries must
be identical.  Each variant runs in a subprocess on the same deterministic model.
"""
import hashlib
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import hashlib, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
import paper_2208_04448_b300 as nv
from fixtures import query_points, workload
ijk, val, _ = workload("sphere128", device="cuda")
g = nv.build(ijk.contiguous(), val.contiguous(), 0, 3.0)
m = nv.compress(g, seed=4, ffm_sigma=1.25, steps=60, batch=4096, width=[32, 64, 64], layers=[3, 4, 4],
                ffm_size=[32, 64], patch_precs=(1 << nv.FP16) | (1 << nv.BF16))
h = hashlib.sha256()
for prec in (nv.FP16, nv.BF16):
    dijk, dval, cnt = nv.decompress(m, prec)
    h.update(dijk.cpu().numpy().tobytes()); h.update(dval.cpu().numpy().tobytes())
    pts = ijk[:5000].contiguous()
    for net in (0, 1, 2):
        h.update(nv.mlp_eval(m, net, pts, prec).cpu().numpy().tobytes())
    q = query_points(ijk.cpu(), 20000, seed=3).cuda()
    out, act = nv.query(m, q, prec, active=True)
    h.update(out.cpu().numpy().tobytes()); h.update(act.cpu().numpy().tobytes())
print("DIGEST", h.hexdigest())
"""


def _digest(variant: int) -> str:
    env = dict(os.environ, NVDB_TC_VARIANT=str(variant))
    code = CHILD.format(root=ROOT)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("DIGEST ")]
    assert lines, r.stdout[-2000:]
    return lines[-1].split()[1]


def test_kernel_variants_give_the_same_bits():
    d = [_digest(v) for v in (0, 1, 2)]
    assert d[0] == d[1] == d[2], d
