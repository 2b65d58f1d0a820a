"""The C-ABI library loads and exports every symbol include/nvdb.h declares (CPU only)."""
import os
import re

from paper_2208_04448_b300 import _native as N

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "nvdb.h")


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
    import ctypes as C
    assert C.sizeof(N.TrainOpts) == 112 and N.TrainOpts.subdomain.offset == 96 and N.TrainOpts.sampling.offset == 108
    assert C.sizeof(N.Info) == 72 and N.Info.n_active.offset == 32 and N.Info.n_experts.offset == 64
    assert C.sizeof(N.BuildOpts) == 8


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
