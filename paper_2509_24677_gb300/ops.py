"""Python binding of the npvs C ABI: one function per entry point, same names, argument
marshalling only (torch tensors -> device pointers, the current CUDA stream). Every step of the
path runs in libnpvs.so; these functions raise NpvsError on a non-OK status.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import torch

from . import _lib as L
from ._lib import NpvsError, check  # noqa: F401  (re-exported)


def _lib():
    return L.load()


def _p(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _s(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("npvs: device tensors required")


class Workspace:
    """A growable device scratch buffer (caller-owned memory handed to the library)."""

    def __init__(self, device="cuda"):
        self.device = device
        self.buf = torch.empty(0, dtype=torch.uint8, device=device)

    def get(self, nbytes: int) -> torch.Tensor:
        if self.buf.numel() < nbytes:
            self.buf = torch.empty(max(nbytes, 2 * self.buf.numel()), dtype=torch.uint8, device=self.device)
        return self.buf


_default_ws = {}


def _ws(ws: Optional[Workspace], nbytes: int) -> torch.Tensor:
    if ws is None:
        dev = torch.cuda.current_device()
        ws = _default_ws.setdefault(dev, Workspace(f"cuda:{dev}"))
    return ws.get(nbytes)


def grid(W, H, D, B=1) -> L.Grid:
    return L.Grid(W, H, D, B)


def dims(X, Y, Z, B=1) -> L.Dims:
    return L.Dims(X, Y, Z, B)


# ---- status / errors ----------------------------------------------------------------------

def npvs_version() -> str:
    return _lib().npvs_version().decode()


def npvs_launch_count() -> int:
    return int(_lib().npvs_launch_count())


def npvs_last_error() -> str:
    return _lib().npvs_last_error().decode()


def npvs_check_status(status: torch.Tensor, stream=None) -> int:
    """Synchronises, returns and clears the device status word (0 = OK)."""
    _need_cuda(status)
    return _lib().npvs_check_status(_p(status), _s(stream))


# ---- a1 ---------------------------------------------------------------------------------------

def npvs_camera_setup(vc, n_slices: int) -> L.Camera:
    """vc: any object with centre, half, yaw, fov_deg, rot_deg, near, far (npvs_inputs.Viewcell)."""
    v = L.Viewcell((ctypes.c_double * 3)(*vc.centre), vc.half, vc.yaw, vc.fov_deg, vc.rot_deg, vc.near, vc.far)
    cam = L.Camera()
    check(_lib().npvs_camera_setup(ctypes.byref(v), n_slices, ctypes.byref(cam)), "npvs_camera_setup")
    return cam


def cameras_to_device(cams: Sequence[L.Camera], device="cuda") -> torch.Tensor:
    raw = b"".join(bytes(c) for c in cams)
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)


# ---- a2 ---------------------------------------------------------------------------------------

def npvs_froxelize(boxes, box_offsets, cams_dev, g: L.Grid, supersample: int, occ_bits,
                   ws: Optional[Workspace] = None, stream=None):
    _need_cuda(boxes, box_offsets, cams_dev, occ_bits)
    n = boxes.shape[0]
    nb = _lib().npvs_froxelize_workspace_bytes(n)
    w = _ws(ws, nb)
    check(_lib().npvs_froxelize(_p(boxes), _p(box_offsets), n, _p(cams_dev), g, supersample, _p(occ_bits),
                                _p(w), w.numel(), _s(stream)), "npvs_froxelize")


# ---- a3 / a7 ----------------------------------------------------------------------------------

def npvs_interleave(occ_bits, g: L.Grid, d: int, in_ch: int, feat_dtype: int, capacity: int, coords, feats,
                    n_active, table=None, status=None, ws: Optional[Workspace] = None, stream=None):
    _need_cuda(occ_bits, coords, feats, n_active, table, status)
    nb = _lib().npvs_interleave_workspace_bytes(g, d)
    w = _ws(ws, nb)
    check(_lib().npvs_interleave(_p(occ_bits), g, d, in_ch, feat_dtype, capacity, _p(coords), _p(feats),
                                 _p(n_active), _p(table), _p(status), _p(w), w.numel(), _s(stream)),
          "npvs_interleave")


def npvs_interleave_noalloc(occ_bits, g: L.Grid, d: int, in_ch: int, feat_dtype: int, capacity: int, coords,
                            feats, n_active, table=None, status=None, stream=None):
    """npvs_interleave without a workspace argument, for callers that cannot allocate device memory:
    the library keeps the scratch in a fixed device array (limit and sharing rules in npvs.h)."""
    _need_cuda(occ_bits, coords, feats, n_active, table, status)
    check(_lib().npvs_interleave_noalloc(_p(occ_bits), g, d, in_ch, feat_dtype, capacity, _p(coords), _p(feats),
                                         _p(n_active), _p(table), _p(status), _s(stream)),
          "npvs_interleave_noalloc")


def npvs_deinterleave(logits, table, n_active, g: L.Grid, d: int, tau: float, mask_bits, pvs_bits,
                      probs_out=None, capacity: int = 0, stream=None):
    _need_cuda(logits, table, n_active, mask_bits, pvs_bits, probs_out)
    check(_lib().npvs_deinterleave(_p(logits), _p(table), _p(n_active), g, d, float(tau), _p(mask_bits),
                                   _p(pvs_bits), _p(probs_out), capacity, _s(stream)), "npvs_deinterleave")


# ---- a4 ---------------------------------------------------------------------------------------

def level_struct(lv) -> L.Level:
    """lv: object with dims (L.Dims), capacity, coords, n_rows, table tensors."""
    return L.Level(lv.dims, lv.capacity, _p(lv.coords), _p(lv.n_rows), _p(lv.table))


def npvs_build_rulebook(kind: int, lv_in, lv_out, map_, map2=None, status=None,
                        ws: Optional[Workspace] = None, stream=None):
    a = level_struct(lv_in)
    b = level_struct(lv_out) if lv_out is not None else None
    nb = _lib().npvs_rulebook_workspace_bytes(lv_out.dims if lv_out is not None else lv_in.dims)
    w = _ws(ws, nb)
    check(_lib().npvs_build_rulebook(kind, ctypes.byref(a), ctypes.byref(b) if b is not None else None,
                                     _p(map_), _p(map2), _p(status), _p(w), w.numel(), _s(stream)),
          "npvs_build_rulebook")


# ---- a5 / a6 ----------------------------------------------------------------------------------

def npvs_packed_weight_bytes(kind: int, cin: int, cout: int) -> int:
    return _lib().npvs_packed_weight_bytes(kind, cin, cout)


def npvs_pack_weights(kind: int, cin: int, cout: int, w32: torch.Tensor, packed: torch.Tensor, stream=None):
    _need_cuda(w32, packed)
    assert w32.dtype == torch.float32 and w32.is_contiguous()
    check(_lib().npvs_pack_weights(kind, cin, cout, _p(w32), _p(packed), _s(stream)), "npvs_pack_weights")


def npvs_conv_workspace_bytes(desc: Optional[L.ConvDesc] = None) -> int:
    return int(_lib().npvs_conv_workspace_bytes(ctypes.byref(desc) if desc is not None else None))


def conv_workspace(nbytes: Optional[int] = None, device="cuda") -> torch.Tensor:
    """A zero-filled BF16-convolution workspace (split-K partials and counters, product tiles)."""
    return torch.zeros(nbytes if nbytes is not None else npvs_conv_workspace_bytes(), dtype=torch.uint8,
                       device=device)


def conv_desc(kind, dtype, cin, cout, relu, map_, n_out, cap_out, out_f32=False, map2=None, n_in=None,
              cap_in=0, status=None, workspace: Optional[torch.Tensor] = None, stages: int = 0,
              max_split: int = 0, lag: int = 0, gather: int = 0, gather_warps: int = 0,
              form: int = 0) -> L.ConvDesc:
    return L.ConvDesc(kind, dtype, cin, cout, int(relu), int(out_f32), _p(map_), _p(map2), _p(n_out), cap_out,
                      _p(n_in), cap_in, _p(status), _p(workspace),
                      0 if workspace is None else workspace.numel(), stages, max_split, lag, gather, gather_warps,
                      form)


def npvs_sparse_conv_fwd(desc: L.ConvDesc, x, w, bias, skip, y, stream=None):
    _need_cuda(x, w, bias, skip, y)
    check(_lib().npvs_sparse_conv_fwd(ctypes.byref(desc), _p(x), _p(w), _p(bias), _p(skip), _p(y), _s(stream)),
          "npvs_sparse_conv_fwd")
