"""Oracle froxelization and ground truth (test infrastructure; see ``oracle/__init__``).

Thin ctypes wrapper over ``oracle/froxel.c``; the arithmetic and its citations live there
(Sec. 3.2: froxelization with supersampling; ground truth by dense viewpoint sampling).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "froxel.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle_froxel.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no floating-point contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.oracle_froxelize.argtypes = [P, P, I, I, I, I, P, I, I, P]
            lib.oracle_froxelize.restype = None
            lib.oracle_froxel_columns.argtypes = [P, P, I, I, I, I, P, I, I, P, I, P]
            lib.oracle_froxel_columns.restype = None
            lib.oracle_slice_of.argtypes = [P, I, ctypes.c_float]
            lib.oracle_slice_of.restype = I
            lib.oracle_ray_dir_f32.argtypes = [P, I, I, I, I, P]
            lib.oracle_ray_dir_f32.restype = None
            lib.oracle_gt_raycast.argtypes = [P, P, I, I, I, I, P, I, P, I, P]
            lib.oracle_gt_raycast.restype = ctypes.c_longlong
            lib.oracle_gt_raycast_f32.argtypes = [P, P, I, I, I, I, P, I, P, I, P]
            lib.oracle_gt_raycast_f32.restype = ctypes.c_longlong
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cam_vec(cam) -> np.ndarray:
    return np.ascontiguousarray(np.concatenate([cam.origin, cam.right, cam.up, cam.fwd,
                                                [cam.tan_half]]).astype(np.float32))


def froxelize(cam, boxes: np.ndarray, W: int, H: int, D: int, s: int, precision: int = 32) -> np.ndarray:
    """Geometry grid G as bits [D][H][W/32] (uint32) for one camera."""
    assert W % 32 == 0 and len(cam.slices) == D + 1
    lib = _load()
    cv = _cam_vec(cam)
    z = np.ascontiguousarray(cam.slices, dtype=np.float32)
    bx = np.ascontiguousarray(boxes, dtype=np.float32)
    bits = np.zeros((D, H, W // 32), dtype=np.uint32)
    lib.oracle_froxelize(_ptr(cv), _ptr(z), W, H, D, s, _ptr(bx), len(bx), precision, _ptr(bits))
    return bits


def froxel_columns(cam, boxes, W, H, D, s, cols: np.ndarray, precision: int = 32) -> np.ndarray:
    """Slice bits of selected froxel columns: cols [n][2] (x, y) -> [n][ceil(D/32)] uint32."""
    lib = _load()
    cv = _cam_vec(cam)
    z = np.ascontiguousarray(cam.slices, dtype=np.float32)
    bx = np.ascontiguousarray(boxes, dtype=np.float32)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros((len(c), (D + 31) // 32), dtype=np.uint32)
    lib.oracle_froxel_columns(_ptr(cv), _ptr(z), W, H, D, s, _ptr(bx), len(bx), precision,
                              _ptr(c), len(c), _ptr(out))
    return out


def prune(cam, boxes: np.ndarray, W: int, H: int, D: int, s: int, pvs_bits: np.ndarray,
          precision: int = 32) -> np.ndarray:
    """Pruning by the PVS. Sec. 3.2: a fragment that falls in a froxel the PVS leaves empty can be
    discarded; Sec. 5.6: a moving object's temporal bounding volume is froxelized and the object is
    dropped when none of its froxels is visible. Definition written out: box i is kept (1) iff the
    froxelization of box i alone shares a froxel with pvs_bits [D][H][W/32]; else 0."""
    out = np.zeros(len(boxes), dtype=np.uint8)
    for i in range(len(boxes)):
        gi = froxelize(cam, boxes[i:i + 1], W, H, D, s, precision)
        out[i] = 1 if np.any(gi & pvs_bits) else 0
    return out


def slice_of(cam, t: float) -> int:
    z = np.ascontiguousarray(cam.slices, dtype=np.float32)
    return _load().oracle_slice_of(_ptr(z), len(z) - 1, float(np.float32(t)))


def ray_dir_f32(cam, a: int, b: int, sW: int, sH: int) -> np.ndarray:
    out = np.zeros(3, dtype=np.float32)
    _load().oracle_ray_dir_f32(_ptr(_cam_vec(cam)), a, b, sW, sH, _ptr(out))
    return out


def points_outside_boxes(pts: np.ndarray, boxes: np.ndarray) -> np.ndarray:
    """Mask of viewpoints that lie inside no box (closed boxes)."""
    b = boxes.astype(np.float64)
    inside = np.zeros(len(pts), dtype=bool)
    for i in range(0, len(b), 512):
        bb = b[i:i + 512]
        ge = (pts[:, None, :] >= bb[None, :, :3]).all(-1)
        le = (pts[:, None, :] <= bb[None, :, 3:]).all(-1)
        inside |= (ge & le).any(-1)
    return ~inside


def gt_raycast(cam, boxes, W, H, D, s_gt: int, pts: np.ndarray, precision: int = 64):
    """Raw ground truth [D][H][W/32] from the given viewpoints (not yet ANDed with G).
    precision 64: binary64 nearest face hit (viewpoints taken as float64); 32: the binary32
    mirror (viewpoints rounded to float32). Returns (bits, number of rays that hit geometry)."""
    lib = _load()
    cv = _cam_vec(cam)
    z = np.ascontiguousarray(cam.slices, dtype=np.float32)
    bx = np.ascontiguousarray(boxes, dtype=np.float32)
    bits = np.zeros((D, H, W // 32), dtype=np.uint32)
    if precision == 32:
        p = np.ascontiguousarray(pts, dtype=np.float32)
        nhit = lib.oracle_gt_raycast_f32(_ptr(cv), _ptr(z), W, H, D, s_gt, _ptr(p), len(p), _ptr(bx),
                                         len(bx), _ptr(bits))
    else:
        p = np.ascontiguousarray(pts, dtype=np.float64)
        nhit = lib.oracle_gt_raycast(_ptr(cv), _ptr(z), W, H, D, s_gt, _ptr(p), len(p), _ptr(bx),
                                     len(bx), _ptr(bits))
    return bits, int(nhit)


def viewpoints(vc, cam, offsets: np.ndarray) -> np.ndarray:
    """World positions c + a r + b u + e f of camera-frame offsets (a, b, e) in the viewcell
    (float64, basis taken from the camera)."""
    c = np.asarray(vc.centre, dtype=np.float64)
    R = np.stack([np.asarray(cam.right, np.float64), np.asarray(cam.up, np.float64),
                  np.asarray(cam.fwd, np.float64)])
    return c[None, :] + np.asarray(offsets, dtype=np.float64) @ R


def ground_truth(vc, cam, boxes, W, H, D, s_gt, offsets: np.ndarray, M: int, G: np.ndarray,
                 precision: int = 64):
    """GT := raw ray-cast PVS from the first M candidate viewpoints outside every box, ANDed with
    the geometry grid G. Reading of Sec. 3.2's occlusion-culling property (supp of the PVS lies
    inside supp(G)). Returns (gt_bits, raw_bits)."""
    cand = viewpoints(vc, cam, offsets)
    ok = points_outside_boxes(cand, boxes)
    pts = cand[ok][:M]
    if len(pts) < M:
        raise ValueError("not enough viewpoints outside the geometry")
    raw, _ = gt_raycast(cam, boxes, W, H, D, s_gt, pts, precision)
    return raw & G, raw
