"""NeuralVDB hot path on B300 -- Python binding of libnvdb.so (include/nvdb.h).

Every function marshals torch CUDA tensors (device pointers) and the current
torch stream into the C ABI; all computation runs in the library's CUDA
kernels.  There is no CPU fallback: the binding raises if libnvdb.so is not
built.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _native as N
from ._native import (BF16, BF16X3, FP16, FP32, FP8_E4M3, INJECT_ALLOC_BUDGET, INJECT_FUSED_ADAM,  # noqa: F401
                      INJECT_STATIC_LIMIT, INJECT_WAIT_TIMEOUT,
                      ERR_CAPACITY, ERR_CORRUPT, ERR_INVALID_ARG, ERR_OUT_OF_MEMORY, ERR_TIMEOUT, ERR_UNSUPPORTED,
                      LOSS_BCE, LOSS_CE, LOSS_L1, LOSS_LINEAR, LOSS_MSE,
                      NET_L0_CLASSIFIER, NET_L1_CLASSIFIER, NET_REGRESSOR, NET_TILE_REGRESSOR, ACT_RELU, ACT_SIN)

_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = N.load()
    return _lib


class NvdbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"nvdb status {status}: {msg}")
        self.status = status


def _check(st: int):
    if st != N.OK:
        raise NvdbError(st, lib().nvdb_last_error().decode())


def _stream(stream=None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t: torch.Tensor, dtype, name: str) -> C.c_void_p:
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    return C.c_void_p(t.data_ptr())


def _info(fn, h) -> dict:
    i = N.Info()
    _check(fn(h, C.byref(i)))
    return dict(grid_class=i.grid_class, background=i.background, half_width=i.half_width,
                origin=list(i.origin), log2_extent=i.log2_extent, n_active=i.n_active, n_leaf=i.n_leaf,
                n_l1=i.n_l1, n_l2=i.n_l2, n_experts=i.n_experts, subdomain=i.subdomain, n_tiles=i.n_tiles)


class Grid:
    """Explicit VDB [Hash,5,4,3] tree on the device (nvdb_grid)."""

    def __init__(self, handle: C.c_void_p):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        return _info(lib().nvdb_grid_info, self._h)

    def read(self) -> dict:
        """Canonical arrays as host numpy arrays."""
        import numpy as np
        i = self.info()
        a = dict(ijk=np.empty((i["n_active"], 3), np.int32), val=np.empty(i["n_active"], np.float32),
                 leaf_origin=np.empty((i["n_leaf"], 3), np.int32), leaf_mask=np.empty((i["n_leaf"], 8), np.uint64),
                 l1_origin=np.empty((i["n_l1"], 3), np.int32), l1_mask=np.empty((i["n_l1"], 64), np.uint64))
        p = [a[k].ctypes.data_as(C.c_void_p) for k in ("ijk", "val", "leaf_origin", "leaf_mask", "l1_origin", "l1_mask")]
        _check(lib().nvdb_grid_read(self._h, *p, _stream()))
        return a

    def tiles(self) -> dict:
        """Active tiles (tile pruning): leaf_tile [n_leaf] bool, l1_tile_mask [n_l1, 64] uint64."""
        import numpy as np
        i = self.info()
        lt = np.empty(i["n_leaf"], np.uint8)
        tm = np.empty((i["n_l1"], 64), np.uint64)
        _check(lib().nvdb_grid_tiles(self._h, lt.ctypes.data_as(C.c_void_p), tm.ctypes.data_as(C.c_void_p), _stream()))
        return dict(leaf_tile=lt.astype(bool), l1_tile_mask=tm)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.nvdb_grid_free(self._h)
            self._h = None


class Model:
    """NeuralVDB [Hash,5,NN(4),NN(3)] model (nvdb_model)."""

    def __init__(self, handle: C.c_void_p):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        return _info(lib().nvdb_model_info, self._h)

    def losses(self, net: int):
        import numpy as np
        n = C.c_int64()
        _check(lib().nvdb_model_losses(self._h, net, None, 0, C.byref(n)))
        out = np.empty(n.value, np.float32)
        _check(lib().nvdb_model_losses(self._h, net, out.ctypes.data_as(C.POINTER(C.c_float)), n.value, None))
        return out

    def param_count(self, net: int) -> int:
        return int(lib().nvdb_net_param_count(self._h, net))

    def params(self, net: int, stream=None) -> torch.Tensor:
        """Flat FP32 parameters of network `net` (a copy on the device, storage order)."""
        out = torch.empty(self.param_count(net), dtype=torch.float32, device="cuda")
        _check(lib().nvdb_net_params(self._h, net, _dptr(out, torch.float32, "params"), _stream(stream)))
        return out

    def set_params(self, net: int, params: torch.Tensor, stream=None):
        """Replace network `net`'s parameters (drops the patch sets until repatch)."""
        if params.numel() != self.param_count(net):
            raise ValueError(f"network {net} has {self.param_count(net)} parameters, got {params.numel()}")
        _check(lib().nvdb_net_set_params(self._h, net, _dptr(params, torch.float32, "params"), _stream(stream)))

    def repatch(self, grid: "Grid", patch_precs: int = 0b11111, stream=None):
        """Patch sets of the current networks against the grid the model encodes."""
        _check(lib().nvdb_model_repatch(self._h, grid.handle, patch_precs, _stream(stream)))

    def export(self) -> bytes:
        n = C.c_size_t()
        _check(lib().nvdb_model_export(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(lib().nvdb_model_export(self._h, buf, C.byref(n)))
        return buf.raw[: n.value]

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.nvdb_model_free(self._h)
            self._h = None


def build(ijk: torch.Tensor, val: torch.Tensor, grid_class: int = 0, half_width: float = 3.0, stream=None,
          prune_tiles: bool = False, tile_tolerance: float = 0.0) -> Grid:
    n = ijk.shape[0]
    o = N.BuildOpts(grid_class, half_width, 1 if prune_tiles else 0, tile_tolerance)
    h = C.c_void_p()
    _check(lib().nvdb_build(_dptr(ijk, torch.int32, "ijk"), _dptr(val, torch.float32, "val"), n, C.byref(o),
                            _stream(stream), C.byref(h)))
    return Grid(h)


def train_opts(**kw) -> N.TrainOpts:
    o = N.TrainOpts()
    lib().nvdb_train_opts_default(C.byref(o))
    for k, v in kw.items():
        if k in ("width", "layers", "ffm_size", "stop_loss"):
            arr = getattr(o, k)
            for i, x in enumerate(v):
                arr[i] = float(x) if k == "stop_loss" else int(x)
        else:
            setattr(o, k, v)
    return o


def compress(grid: Grid, opts=None, warm: "Model | None" = None, stream=None, **kw) -> Model:
    o = opts if opts is not None else train_opts(**kw)
    h = C.c_void_p()
    _check(lib().nvdb_compress(grid.handle, C.byref(o), warm.handle if warm else None, _stream(stream), C.byref(h)))
    return Model(h)


def compress_sequence(grids, refine_lr_scale: float = 0.01, refine_steps: int = 0, warm_steps: int = 500,
                      opts=None, stream=None, **kw) -> list:
    """nvdb_compress_sequence: frame 0 cold (then refined at lr x refine_lr_scale), every later
    frame warm-started from the previous one with the early stop at frame 0's final loss."""
    o = opts if opts is not None else train_opts(**kw)
    arr = (C.c_void_p * len(grids))(*[g.handle for g in grids])
    out = (C.c_void_p * len(grids))()
    _check(lib().nvdb_compress_sequence(arr, len(grids), C.byref(o), refine_lr_scale, refine_steps, warm_steps,
                                        _stream(stream), out))
    return [Model(C.c_void_p(h)) for h in out]


def decompress(models, prec: int = FP32, out=None, stream=None):
    """Decode models -> (ijk int32 [n,3], val float32 [n], counts list).  `out` = (ijk, val) to reuse buffers."""
    if isinstance(models, Model):
        models = [models]
    arr = (C.c_void_p * len(models))(*[m.handle for m in models])
    counts = (C.c_int64 * len(models))()
    _check(lib().nvdb_decompress(arr, len(models), prec, None, None, 0, counts, _stream(stream)))
    total = sum(counts)
    if out is None:
        ijk = torch.empty((total, 3), dtype=torch.int32, device="cuda")
        val = torch.empty(total, dtype=torch.float32, device="cuda")
    else:
        ijk, val = out
    _check(lib().nvdb_decompress(arr, len(models), prec, _dptr(ijk, torch.int32, "ijk"),
                                 _dptr(val, torch.float32, "val"), ijk.shape[0], counts, _stream(stream)))
    return ijk[:total], val[:total], list(counts)


def decompress_host(models, prec: int = FP32, host=None, out=None, stream=None):
    """Decode models into device buffers and, overlapped with the regression, into host
    buffers (nvdb_decompress_host).  `host` = (ijk int32 [n,3], val float32 [n]) CPU
    tensors, pinned for asynchronous copies (allocated pinned if None); `out` = device
    buffers to reuse.  Returns (host ijk, host val, counts)."""
    if isinstance(models, Model):
        models = [models]
    arr = (C.c_void_p * len(models))(*[m.handle for m in models])
    counts = (C.c_int64 * len(models))()
    _check(lib().nvdb_decompress_host(arr, len(models), prec, None, None, None, None, 0, counts, _stream(stream)))
    total = sum(counts)
    ijk, val = out if out is not None else (torch.empty((total, 3), dtype=torch.int32, device="cuda"),
                                            torch.empty(total, dtype=torch.float32, device="cuda"))
    if host is None:
        host = (torch.empty((total, 3), dtype=torch.int32, pin_memory=True),
                torch.empty(total, dtype=torch.float32, pin_memory=True))
    h_ijk, h_val = host
    for h, dt, nm in ((h_ijk, torch.int32, "host ijk"), (h_val, torch.float32, "host val")):
        if h.device.type != "cpu" or h.dtype != dt or not h.is_contiguous() or h.shape[0] < total:
            raise ValueError(f"{nm}: need a contiguous CPU {dt} tensor of at least {total} rows")
    cap = min(ijk.shape[0], h_ijk.shape[0], h_val.shape[0])
    _check(lib().nvdb_decompress_host(arr, len(models), prec, _dptr(ijk, torch.int32, "ijk"),
                                      _dptr(val, torch.float32, "val"), h_ijk.data_ptr(), h_val.data_ptr(), cap,
                                      counts, _stream(stream)))
    return h_ijk[:total], h_val[:total], list(counts)


class Plan:
    """A graph-captured decode of fixed models into fixed output buffers (nvdb_plan)."""

    def __init__(self, handle, models, ijk, val):
        self._h, self._keep = handle, (models, ijk, val)   # keep models and outputs alive
        self.ijk, self.val = ijk, val

    def launch(self, stream=None):
        _check(lib().nvdb_plan_launch(self._h, _stream(stream)))

    def check(self, stream=None):
        _check(lib().nvdb_plan_check(self._h, _stream(stream)))

    def info(self) -> dict:
        occ, var, ms = C.c_int(), C.c_int(), C.c_float()
        _check(lib().nvdb_plan_info(self._h, C.byref(occ), C.byref(var), C.byref(ms)))
        return dict(tc_ctas_per_sm=occ.value, tc_variant=var.value, tuned_ms=ms.value)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.nvdb_plan_free(self._h)
            self._h = None


def decompress_plan(models, prec: int = FP32, stream=None) -> Plan:
    if isinstance(models, Model):
        models = [models]
    arr = (C.c_void_p * len(models))(*[m.handle for m in models])
    counts = (C.c_int64 * len(models))()
    _check(lib().nvdb_decompress(arr, len(models), prec, None, None, 0, counts, _stream(stream)))
    total = sum(counts)
    ijk = torch.empty((total, 3), dtype=torch.int32, device="cuda")
    val = torch.empty(total, dtype=torch.float32, device="cuda")
    h = C.c_void_p()
    _check(lib().nvdb_decompress_plan(arr, len(models), prec, _dptr(ijk, torch.int32, "ijk"),
                                      _dptr(val, torch.float32, "val"), total, _stream(stream), C.byref(h)))
    return Plan(h, list(models), ijk, val)


def query(model: Model, xyz: torch.Tensor, prec: int = FP32, active: bool = False, out=None, stream=None):
    n = xyz.shape[0]
    res = out if out is not None else torch.empty(n, dtype=torch.float32, device="cuda")
    act = torch.empty(n, dtype=torch.uint8, device="cuda") if active else None
    _check(lib().nvdb_query(model.handle, _dptr(xyz, torch.float32, "xyz"), n, prec, _dptr(res, torch.float32, "out"),
                            _dptr(act, torch.uint8, "active") if act is not None else None, _stream(stream)))
    return (res, act) if active else res


def grid_sample(grid: Grid, xyz: torch.Tensor, order: int = 1, out=None, stream=None) -> torch.Tensor:
    """nvdb_grid_sample: order-0 / 1 / 3 point samples of the explicit grid."""
    n = xyz.shape[0]
    res = out if out is not None else torch.empty(n, dtype=torch.float32, device="cuda")
    _check(lib().nvdb_grid_sample(grid.handle, _dptr(xyz, torch.float32, "xyz"), n, order,
                                  _dptr(res, torch.float32, "out"), _stream(stream)))
    return res


def grid_isosurface(grid: Grid, stream=None) -> torch.Tensor:
    """nvdb_grid_isosurface: the level set's zero crossings along voxel edges, float [m, 3]."""
    cnt = C.c_int64()
    _check(lib().nvdb_grid_isosurface(grid.handle, None, 0, C.byref(cnt), _stream(stream)))
    pts = torch.empty((cnt.value, 3), dtype=torch.float32, device="cuda")
    if cnt.value:
        _check(lib().nvdb_grid_isosurface(grid.handle, _dptr(pts, torch.float32, "pts"), cnt.value, C.byref(cnt),
                                          _stream(stream)))
    return pts


def mcd(reference: Grid, reconstruction: Grid, stream=None) -> float:
    """nvdb_mcd: modified Chamfer distance (Eq. 4) between two level-set grids, in voxels."""
    v = C.c_double()
    _check(lib().nvdb_mcd(reference.handle, reconstruction.handle, C.byref(v), _stream(stream)))
    return v.value


def render(model: Model, eye, target, up=(0.0, 1.0, 0.0), fov_deg: float = 40.0, width: int = 256, height: int = 256,
           step: float = 1.0, max_steps: int = 512, sigma: float = 0.05, prec: int = FP32, out=None,
           stream=None) -> torch.Tensor:
    """nvdb_render: ray-marched (radiance, transmittance) image [height, width, 2] on the device."""
    cam = N.Camera()
    cam.eye[:], cam.target[:], cam.up[:] = [float(v) for v in eye], [float(v) for v in target], [float(v) for v in up]
    cam.fov_deg, cam.width, cam.height, cam.step, cam.max_steps, cam.sigma = fov_deg, width, height, step, max_steps, sigma
    img = out if out is not None else torch.empty((height, width, 2), dtype=torch.float32, device="cuda")
    _check(lib().nvdb_render(model.handle, C.byref(cam), prec, _dptr(img, torch.float32, "image"), _stream(stream)))
    return img


def mlp_eval(model: Model, net: int, ijk: torch.Tensor, prec: int = FP32, stream=None) -> torch.Tensor:
    """Raw network outputs at voxel coordinates ([n]; [n, 3] logits for the ternary level-1
    classifier of a model with active tiles)."""
    n = ijk.shape[0]
    wide = net == 0 and model.info()["n_tiles"] > 0
    out = torch.empty((n, 3) if wide else n, dtype=torch.float32, device="cuda")
    _check(lib().nvdb_mlp_eval(model.handle, net, prec, _dptr(ijk, torch.int32, "ijk"), n,
                               _dptr(out, torch.float32, "out"), _stream(stream)))
    return out


def check_grad_args(param_count: int, ijk: torch.Tensor, target: torch.Tensor, out=None) -> int:
    """Shapes of a gradient call, checked before anything is launched: ijk [n, 3], target [n],
    out (if given) exactly param_count elements.  Returns n."""
    if ijk.dim() != 2 or ijk.shape[1] != 3:
        raise ValueError(f"ijk must be [n, 3], got {tuple(ijk.shape)}")
    n = ijk.shape[0]
    if target.numel() != n:
        raise ValueError(f"target must hold n = {n} values, got {target.numel()}")
    if out is not None and out.numel() != param_count:
        raise ValueError(f"out must hold param_count = {param_count} floats, got {out.numel()}")
    return n


def mlp_grad(model: Model, net: int, ijk: torch.Tensor, target: torch.Tensor, loss: int, prec: int = FP32,
             stream=None):
    """nvdb_mlp_grad: (gradient [param_count(net)], mean loss).  The ternary level-1 classifier
    takes loss=LOSS_CE with class targets 0, 1, 2 (as floats); the other networks any other loss."""
    check_grad_args(model.param_count(net), ijk, target)
    g = torch.empty(model.param_count(net), dtype=torch.float32, device="cuda")
    lv = C.c_float()
    _check(lib().nvdb_mlp_grad(model.handle, net, prec, _dptr(ijk, torch.int32, "ijk"),
                               _dptr(target, torch.float32, "target"), ijk.shape[0], loss,
                               _dptr(g, torch.float32, "grad"), C.byref(lv), _stream(stream)))
    return g, lv.value


def mlp_grad_static(model: Model, net: int, ijk: torch.Tensor, target: torch.Tensor, loss: int, out=None,
                    stream=None):
    """nvdb_mlp_grad_static: the gradient of mlp_grad computed without any device allocation by the
    library.  `out` (a float32 CUDA tensor of param_count(net) elements) lets the caller own the output too."""
    check_grad_args(model.param_count(net), ijk, target, out)
    g = out if out is not None else torch.empty(model.param_count(net), dtype=torch.float32, device="cuda")
    lv = C.c_float()
    _check(lib().nvdb_mlp_grad_static(model.handle, net, _dptr(ijk, torch.int32, "ijk"),
                                      _dptr(target, torch.float32, "target"), ijk.shape[0], loss,
                                      _dptr(g, torch.float32, "grad"), C.byref(lv), _stream(stream)))
    return g, lv.value


class NetworkFunction(torch.autograd.Function):
    """y = network `net` of `model` at voxel coordinates ijk (int32 [n, 3]; leaf units for
    the level-1 classifier as in mlp_eval), differentiable in the network's flat FP32
    parameters.  Forward: the parameters go into the model, then the network kernel
    (nvdb_mlp_eval).  Backward: the hand-written gradient kernel with the upstream dL/dy as
    its linear loss (nvdb_mlp_grad, NVDB_LOSS_LINEAR), in the arithmetic of `prec` (FP32, or
    BF16 on the tensor cores).  Coordinates get no gradient."""

    @staticmethod
    def forward(ctx, params: torch.Tensor, model: Model, net: int, ijk: torch.Tensor, prec: int = FP32):
        if prec not in (FP32, BF16):
            raise ValueError("NetworkFunction: precision FP32 or BF16")
        model.set_params(net, params.detach().contiguous())
        ctx.model, ctx.net, ctx.prec = model, net, prec
        ctx.save_for_backward(ijk)
        return mlp_eval(model, net, ijk, prec)

    @staticmethod
    def backward(ctx, grad_y: torch.Tensor):
        (ijk,) = ctx.saved_tensors
        g, _ = mlp_grad(ctx.model, ctx.net, ijk, grad_y.detach().float().contiguous(), LOSS_LINEAR, ctx.prec)
        return g, None, None, None, None


def network(params: torch.Tensor, model: Model, net: int, ijk: torch.Tensor, prec: int = FP32) -> torch.Tensor:
    """NetworkFunction.apply: network `net` as a differentiable function of `params`."""
    return NetworkFunction.apply(params, model, net, ijk, prec)


def model_import(blob, stream=None) -> Model:
    """nvdb_model_import from `bytes` or from a contiguous uint8 CPU tensor (pass a pinned
    one to make the host-to-device copies direct); the buffer is read, not copied first."""
    h = C.c_void_p()
    if isinstance(blob, torch.Tensor):
        if blob.device.type != "cpu" or blob.dtype != torch.uint8 or not blob.is_contiguous():
            raise ValueError("model_import: a contiguous uint8 CPU tensor")
        ptr, n = C.c_void_p(blob.data_ptr()), blob.numel()
    else:
        ptr, n = bytes(blob), len(blob)
    _check(lib().nvdb_model_import(ptr, n, _stream(stream), C.byref(h)))
    return Model(h)


def debug_inject(what: int, value: int):
    """nvdb_debug_inject: fault injection for tests (INJECT_WAIT_TIMEOUT, INJECT_ALLOC_BUDGET,
    INJECT_STATIC_LIMIT)."""
    _check(lib().nvdb_debug_inject(what, value))


def debug_wait_selftest(limit_ns: int):
    """nvdb_debug_wait_selftest: a bounded wait that runs out (raises NvdbError TIMEOUT)."""
    _check(lib().nvdb_debug_wait_selftest(limit_ns))


def profile_enable(on: bool = True):
    lib().nvdb_profile_enable(1 if on else 0)


def profile_read() -> dict:
    """{kernel name: (launches, total ms)} of the launches recorded since the last read."""
    cap, nl = 64, 64
    names = C.create_string_buffer(cap * nl)
    la = (C.c_int64 * cap)()
    ms = (C.c_double * cap)()
    n = lib().nvdb_profile_read(names, nl, la, ms, cap)
    out = {}
    for i in range(min(n, cap)):
        nm = names.raw[i * nl:(i + 1) * nl].split(b"\0", 1)[0].decode()
        out[nm] = (int(la[i]), float(ms[i]))
    return out


def launch_count() -> int:
    return int(lib().nvdb_launch_count())
