"""ctypes view of include/npvs.h and the loader of the in-tree libnpvs.so.

Loading fails loudly (ImportError) when the library is missing or cannot be loaded; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

NPVS_MAX_SLICES = 256

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CAPACITY, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT = range(7)
F32, BF16, F64 = 0, 1, 2
RB_SUBM3, RB_DOWN2, RB_SUBM3_TABLE, RB_DOWN3 = 0, 1, 2, 3
CONV_SUBM3, CONV_DOWN2, CONV_UP2, CONV_HEAD1, CONV_DOWN3, CONV_UP3 = 0, 1, 2, 3, 4, 5

STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "CAPACITY", 4: "WORKSPACE",
                5: "CUDA", 6: "TIMEOUT"}

P = ctypes.c_void_p
I32 = ctypes.c_int32
SZ = ctypes.c_size_t


class Grid(ctypes.Structure):
    _fields_ = [("W", I32), ("H", I32), ("D", I32), ("B", I32)]


class Dims(ctypes.Structure):
    _fields_ = [("X", I32), ("Y", I32), ("Z", I32), ("B", I32)]


class Viewcell(ctypes.Structure):
    _fields_ = [("centre", ctypes.c_double * 3), ("half_size", ctypes.c_double), ("yaw", ctypes.c_double),
                ("fov_deg", ctypes.c_double), ("rot_deg", ctypes.c_double), ("near_", ctypes.c_double),
                ("far_", ctypes.c_double)]


class Camera(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("right", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("fwd", ctypes.c_float * 3), ("tan_half", ctypes.c_float), ("n_slices", I32),
                ("slices", ctypes.c_float * (NPVS_MAX_SLICES + 1))]


class Level(ctypes.Structure):
    _fields_ = [("dims", Dims), ("capacity", I32), ("coords", P), ("n_rows", P), ("table", P)]


class ConvDesc(ctypes.Structure):
    _fields_ = [("kind", I32), ("dtype", I32), ("cin", I32), ("cout", I32), ("relu", I32), ("out_f32", I32),
                ("map", P), ("map2", P), ("n_out", P), ("cap_out", I32), ("n_in", P), ("cap_in", I32),
                ("status", P), ("workspace", P), ("workspace_bytes", SZ), ("tune_stages", I32),
                ("tune_max_split", I32), ("tune_lag", I32), ("tune_gather", I32), ("tune_gather_warps", I32),
                ("tune_form", I32), ("w_transposed", P)]


class PackJob(ctypes.Structure):
    _fields_ = [("kind", I32), ("cin", I32), ("cout", I32), ("transposed", I32), ("w", P), ("packed", P)]


class LossParams(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("eps", ctypes.c_double), ("lam", ctypes.c_double),
                ("w_bce", ctypes.c_double)]


class AdamParams(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("weight_decay", ctypes.c_float)]


class NetLayer(ctypes.Structure):
    _fields_ = [("kind", I32), ("cin", I32), ("cout", I32), ("relu", I32), ("w", P), ("bias", P),
                ("tune_stages", I32), ("tune_max_split", I32), ("tune_lag", I32), ("tune_gather", I32),
                ("tune_gather_warps", I32), ("tune_form", I32)]


class NetDesc(ctypes.Structure):
    _fields_ = [("grid", Grid), ("d", I32), ("in_ch", I32), ("supersample", I32), ("dtype", I32),
                ("tau", ctypes.c_float), ("max_boxes", I32), ("capacity_permille", I32), ("n_layers", I32),
                ("layers", ctypes.POINTER(NetLayer)), ("chain_level", I32)]


LOSS_TERMS = 12
(LT_L, LT_DICE, LT_ATTR, LT_REP, LT_BCE, LT_GTP, LT_TP, LT_FN, LT_FP, LT_NOCC, LT_DTP,
 LT_DFP) = range(LOSS_TERMS)

# name -> (restype, argtypes)
SIGNATURES = {
    "npvs_last_error": (ctypes.c_char_p, []),
    "npvs_version": (ctypes.c_char_p, []),
    "npvs_launch_count": (ctypes.c_ulonglong, []),
    "npvs_check_status": (I32, [P, P]),
    "npvs_set_wait_limit": (I32, [ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "npvs_camera_setup": (I32, [ctypes.POINTER(Viewcell), I32, ctypes.POINTER(Camera)]),
    "npvs_froxelize_workspace_bytes": (SZ, [I32]),
    "npvs_froxelize": (I32, [P, P, I32, P, Grid, I32, P, P, SZ, P]),
    "npvs_prune": (I32, [P, P, I32, P, Grid, I32, P, P, P, SZ, P]),
    "npvs_interleave_workspace_bytes": (SZ, [Grid, I32]),
    "npvs_interleave": (I32, [P, Grid, I32, I32, I32, I32, P, P, P, P, P, P, SZ, P]),
    "npvs_interleave_noalloc": (I32, [P, Grid, I32, I32, I32, I32, P, P, P, P, P, P]),
    "npvs_deinterleave": (I32, [P, P, P, Grid, I32, ctypes.c_float, P, P, P, I32, P]),
    "npvs_rulebook_workspace_bytes": (SZ, [Dims]),
    "npvs_build_rulebook": (I32, [I32, ctypes.POINTER(Level), ctypes.POINTER(Level), P, P, P, P, SZ, P]),
    "npvs_conv_workspace_bytes": (SZ, [ctypes.POINTER(ConvDesc)]),
    "npvs_packed_weight_bytes": (SZ, [I32, I32, I32]),
    "npvs_pack_weights": (I32, [I32, I32, I32, P, P, P]),
    "npvs_packed_weight_bytes_transposed": (SZ, [I32, I32, I32]),
    "npvs_pack_weights_many": (I32, [I32, ctypes.POINTER(PackJob), P]),
    "npvs_sparse_conv_fwd": (I32, [ctypes.POINTER(ConvDesc), P, P, P, P, P, P]),
    "npvs_gt_raycast": (I32, [P, P, P, P, I32, Grid, I32, P, P, P]),
    "npvs_forward_workspace_bytes": (SZ, [ctypes.POINTER(NetDesc)]),
    "npvs_forward": (I32, [ctypes.POINTER(NetDesc), P, P, I32, P, P, P, P, P, P, SZ, P]),
    "npvs_forward_layer_output": (I32, [ctypes.POINTER(NetDesc), I32, P, ctypes.POINTER(P),
                                        ctypes.POINTER(I32), ctypes.POINTER(P)]),
    "npvs_conv_bwd_workspace_bytes": (SZ, [ctypes.POINTER(ConvDesc)]),
    "npvs_sparse_conv_bwd": (I32, [ctypes.POINTER(ConvDesc), P, P, P, P, P, P, P, P, P, SZ, P]),
    "npvs_loss_workspace_bytes": (SZ, [I32, I32]),
    "npvs_loss_fwd": (I32, [I32, P, P, P, I32, P, P, Grid, I32, ctypes.POINTER(LossParams), P, P, P, SZ, P]),
    "npvs_loss_bwd": (I32, [I32, P, P, P, I32, P, P, Grid, I32, ctypes.POINTER(LossParams), P, P, I32, P, P]),
    "npvs_adam_step": (I32, [P, P, P, P, ctypes.c_int64, ctypes.POINTER(AdamParams), P, P]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libnpvs.so (building it first if it is missing and nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if build_if_missing and (not os.path.exists(path) or _build._stale()):
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libnpvs.so not found at {path}; run paper_2509_24677_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class NpvsError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str):
    if status != OK:
        raise NpvsError(status, where, load().npvs_last_error().decode())
