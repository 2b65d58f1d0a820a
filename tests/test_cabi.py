"""The C-ABI library loads and exports every symbol include/nvdb.h declares (CPU only)."""
import os
import re

from paper_2208_04448_b300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "nvdb.h")


def _declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nvdb_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert sorted(N.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol():
    lib = N.load()
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_layouts():
    """The ctypes structs agree field by field with the C compiler's layout of include/nvdb.h."""
    import ctypes as C
    import shutil
    import subprocess
    import tempfile
    structs = {"nvdb_train_opts": N.TrainOpts, "nvdb_info": N.Info, "nvdb_build_opts": N.BuildOpts,
               "nvdb_camera": N.Camera}
    assert C.sizeof(N.TrainOpts) == 128 and C.sizeof(N.Info) == 80 and C.sizeof(N.BuildOpts) == 16
    gcc = shutil.which("gcc")
    if gcc is None:
        return
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nvdb.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        with open(src, "w") as fh:
            fh.write("\n".join(lines))
        subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_gradient_arguments_rejected_before_any_launch():
    """A short `out`, or ijk / target of the wrong shape, raise before the library is called
    (a short out would otherwise be written past its end on the device)."""
    import pytest
    import torch

    import paper_2208_04448_b300 as nv
    ijk = torch.zeros((10, 3), dtype=torch.int32)
    tgt = torch.zeros(10)
    assert nv.check_grad_args(100, ijk, tgt, torch.zeros(100)) == 10
    with pytest.raises(ValueError, match="out must hold"):
        nv.check_grad_args(100, ijk, tgt, torch.zeros(99))
    with pytest.raises(ValueError, match="target must hold"):
        nv.check_grad_args(100, ijk, torch.zeros(9))
    with pytest.raises(ValueError, match="ijk must be"):
        nv.check_grad_args(100, torch.zeros((10, 2), dtype=torch.int32), tgt)
