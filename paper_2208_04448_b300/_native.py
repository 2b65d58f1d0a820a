"""ctypes declarations of the C ABI in include/nvdb.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnvdb.so")

OK, ERR_INVALID_ARG, ERR_DUPLICATE_VOXEL, ERR_OUT_OF_MEMORY, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, \
    ERR_UNSUPPORTED, ERR_CORRUPT = range(9)
FP32, BF16, FP8_E4M3, FP16, BF16X3 = 0, 1, 2, 3, 4
NET_L1_CLASSIFIER, NET_L0_CLASSIFIER, NET_REGRESSOR, NET_TILE_REGRESSOR = 0, 1, 2, 3
ACT_RELU, ACT_SIN = 0, 1
LOSS_MSE, LOSS_L1, LOSS_BCE, LOSS_LINEAR, LOSS_CE = 0, 1, 2, 3, 4
INJECT_WAIT_TIMEOUT, INJECT_ALLOC_BUDGET, INJECT_STATIC_LIMIT, INJECT_FUSED_ADAM = 1, 2, 3, 4


class BuildOpts(C.Structure):
    _fields_ = [("grid_class", C.c_int32), ("half_width", C.c_float), ("prune_tiles", C.c_int32),
                ("tile_tolerance", C.c_float)]


class TrainOpts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("width", C.c_int32 * 3), ("layers", C.c_int32 * 3),
                ("ffm_size", C.c_int32 * 2), ("ffm_sigma", C.c_float), ("steps", C.c_int32),
                ("batch", C.c_int32), ("lr", C.c_float), ("lr_decay", C.c_float), ("lr_interval", C.c_int32),
                ("loss", C.c_int32), ("train_prec", C.c_int32), ("patch_precs", C.c_uint32),
                ("stop_window", C.c_int32), ("stop_loss", C.c_float * 3), ("resume", C.c_int32),
                ("subdomain", C.c_int32), ("halo", C.c_int32), ("resample", C.c_int32), ("sampling", C.c_int32),
                ("activation", C.c_int32), ("omega", C.c_float), ("tile_width", C.c_int32), ("tile_layers", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("grid_class", C.c_int32), ("background", C.c_float), ("half_width", C.c_float),
                ("origin", C.c_int32 * 3), ("log2_extent", C.c_int32), ("n_active", C.c_int64),
                ("n_leaf", C.c_int64), ("n_l1", C.c_int64), ("n_l2", C.c_int64), ("n_experts", C.c_int32),
                ("subdomain", C.c_int32), ("n_tiles", C.c_int64)]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3), ("fov_deg", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32), ("step", C.c_float), ("max_steps", C.c_int32),
                ("sigma", C.c_float)]


_vp, _i64, _i32, _f32p, _st = C.c_void_p, C.c_int64, C.c_int, C.POINTER(C.c_float), C.c_int

# every symbol include/nvdb.h declares, with its signature
SIGNATURES = {
    "nvdb_build": ([_vp, _vp, _i64, C.POINTER(BuildOpts), _vp, C.POINTER(_vp)], _st),
    "nvdb_grid_info": ([_vp, C.POINTER(Info)], _st),
    "nvdb_grid_read": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _st),
    "nvdb_grid_tiles": ([_vp, _vp, _vp, _vp], _st),
    "nvdb_grid_free": ([_vp], _st),
    "nvdb_train_opts_default": ([C.POINTER(TrainOpts)], None),
    "nvdb_compress": ([_vp, C.POINTER(TrainOpts), _vp, _vp, C.POINTER(_vp)], _st),
    "nvdb_compress_sequence": ([C.POINTER(_vp), _i32, C.POINTER(TrainOpts), C.c_float, C.c_int32, C.c_int32, _vp,
                                C.POINTER(_vp)], _st),
    "nvdb_render": ([_vp, C.POINTER(Camera), _i32, _vp, _vp], _st),
    "nvdb_grid_sample": ([_vp, _vp, _i64, _i32, _vp, _vp], _st),
    "nvdb_grid_isosurface": ([_vp, _vp, _i64, C.POINTER(C.c_int64), _vp], _st),
    "nvdb_mcd": ([_vp, _vp, C.POINTER(C.c_double), _vp], _st),
    "nvdb_model_losses": ([_vp, _i32, _f32p, _i64, C.POINTER(C.c_int64)], _st),
    "nvdb_decompress": ([C.POINTER(_vp), _i32, _i32, _vp, _vp, _i64, C.POINTER(C.c_int64), _vp], _st),
    "nvdb_decompress_host": ([C.POINTER(_vp), _i32, _i32, _vp, _vp, _vp, _vp, _i64, C.POINTER(C.c_int64), _vp], _st),
    "nvdb_decompress_plan": ([C.POINTER(_vp), _i32, _i32, _vp, _vp, _i64, _vp, C.POINTER(_vp)], _st),
    "nvdb_plan_launch": ([_vp, _vp], _st),
    "nvdb_plan_check": ([_vp, _vp], _st),
    "nvdb_plan_info": ([_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_float)], _st),
    "nvdb_plan_free": ([_vp], _st),
    "nvdb_query": ([_vp, _vp, _i64, _i32, _vp, _vp, _vp], _st),
    "nvdb_mlp_eval": ([_vp, _i32, _i32, _vp, _i64, _vp, _vp], _st),
    "nvdb_mlp_grad": ([_vp, _i32, _i32, _vp, _vp, _i64, _i32, _vp, _f32p, _vp], _st),
    "nvdb_mlp_grad_static": ([_vp, _i32, _vp, _vp, _i64, _i32, _vp, _f32p, _vp], _st),
    "nvdb_net_params": ([_vp, _i32, _vp, _vp], _st),
    "nvdb_net_set_params": ([_vp, _i32, _vp, _vp], _st),
    "nvdb_model_repatch": ([_vp, _vp, C.c_uint32, _vp], _st),
    "nvdb_debug_inject": ([_i32, _i64], _st),
    "nvdb_debug_wait_selftest": ([_i64], _st),
    "nvdb_net_param_count": ([_vp, _i32], C.c_int64),
    "nvdb_model_info": ([_vp, C.POINTER(Info)], _st),
    "nvdb_model_export": ([_vp, _vp, C.POINTER(C.c_size_t)], _st),
    "nvdb_model_import": ([_vp, C.c_size_t, _vp, C.POINTER(_vp)], _st),
    "nvdb_model_free": ([_vp], _st),
    "nvdb_last_error": ([], C.c_char_p),
    "nvdb_profile_enable": ([_i32], None),
    "nvdb_profile_read": ([C.c_char_p, _i32, C.POINTER(C.c_int64), C.POINTER(C.c_double), _i32], _i32),
    "nvdb_launch_count": ([], C.c_int64),
}
EXPORTS = list(SIGNATURES)


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"libnvdb.so not built ({path}); run `python -m paper_2208_04448_b300._build`")
    lib = C.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib
