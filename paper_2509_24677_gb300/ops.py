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
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("npvs: tensors passed to the library must be contiguous (row-major)")
    return ctypes.c_void_p(t.data_ptr())


def _s(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


_TDT = {L.F32: torch.float32, L.BF16: torch.bfloat16, L.F64: torch.float64}


def _want(dt, **tensors):
    """Raises TypeError unless every given tensor (None allowed) has torch dtype dt."""
    for name, t in tensors.items():
        if t is not None and t.dtype != dt:
            raise TypeError(f"npvs: {name} must be {dt}, got {t.dtype}")


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


def npvs_set_wait_limit(cycles: int) -> int:
    """Sets the bound (SM cycles; 0 = the default) of the tensor-core kernels' waits for kernels
    launched from now on; returns the previous bound."""
    prev = ctypes.c_int64()
    check(_lib().npvs_set_wait_limit(int(cycles), ctypes.byref(prev)), "npvs_set_wait_limit")
    return int(prev.value)


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


def npvs_prune(boxes, box_offsets, cams_dev, g: L.Grid, supersample: int, pvs_bits, visible,
               ws: Optional[Workspace] = None, stream=None):
    """visible[i] (uint8) = box i's own froxels meet the PVS of its batch element."""
    _need_cuda(boxes, box_offsets, cams_dev, pvs_bits, visible)
    _want(torch.uint8, visible=visible)
    n = boxes.shape[0]
    if visible.numel() < n:
        raise ValueError("npvs_prune: visible needs one byte per box")
    nb = _lib().npvs_froxelize_workspace_bytes(n)
    w = _ws(ws, nb)
    check(_lib().npvs_prune(_p(boxes), _p(box_offsets), n, _p(cams_dev), g, supersample, _p(pvs_bits),
                            _p(visible), _p(w), w.numel(), _s(stream)), "npvs_prune")


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


def npvs_packed_weight_bytes_transposed(kind: int, cin: int, cout: int) -> int:
    return _lib().npvs_packed_weight_bytes_transposed(kind, cin, cout)


def make_pack_jobs(jobs):
    """A host array of npvs_pack_job from (kind, cin, cout, transposed, w32, packed) tuples; the
    tensors must stay alive while the array is used."""
    arr = (L.PackJob * max(1, len(jobs)))()
    for i, (kind, cin, cout, transposed, w32, packed) in enumerate(jobs):
        _need_cuda(w32, packed)
        assert w32.dtype == torch.float32 and w32.is_contiguous()
        arr[i] = L.PackJob(kind, cin, cout, int(transposed), _p(w32), _p(packed))
    return arr, len(jobs)


def npvs_pack_weights_many(jobs, stream=None):
    """jobs: the pair make_pack_jobs returns (or a list of its tuples)."""
    if isinstance(jobs, list):
        jobs = make_pack_jobs(jobs)
    arr, n = jobs
    check(_lib().npvs_pack_weights_many(n, arr, _s(stream)), "npvs_pack_weights_many")


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
    T = _TDT[desc.dtype]
    _want(T, x=x, skip=skip)
    _want(torch.float32 if (desc.out_f32 and desc.dtype != L.F64) else T, y=y)
    _want(torch.float64 if desc.dtype == L.F64 else torch.float32, bias=bias)
    if desc.dtype != L.BF16:
        _want(T, w=w)
    check(_lib().npvs_sparse_conv_fwd(ctypes.byref(desc), _p(x), _p(w), _p(bias), _p(skip), _p(y), _s(stream)),
          "npvs_sparse_conv_fwd")


# ---- the whole frame ---------------------------------------------------------------------------

def npvs_forward_workspace_bytes(net: L.NetDesc) -> int:
    return int(_lib().npvs_forward_workspace_bytes(ctypes.byref(net)))


def npvs_forward(net: L.NetDesc, boxes, box_offsets, n_boxes: int, cams_dev, occ_bits, pvs_bits, probs, status,
                 workspace, stream=None):
    _need_cuda(boxes, box_offsets, cams_dev, occ_bits, pvs_bits, probs, status, workspace)
    _want(torch.float32, boxes=boxes, probs=probs)
    check(_lib().npvs_forward(ctypes.byref(net), _p(boxes), _p(box_offsets), n_boxes, _p(cams_dev), _p(occ_bits),
                              _p(pvs_bits), _p(probs), _p(status), _p(workspace),
                              workspace.numel() * workspace.element_size(), _s(stream)), "npvs_forward")


def npvs_forward_layer_output(net: L.NetDesc, layer: int, workspace):
    """(byte offset into workspace, level capacity, byte offset of the level's row count)."""
    rows, n_rows = ctypes.c_void_p(), ctypes.c_void_p()
    cap = ctypes.c_int32()
    check(_lib().npvs_forward_layer_output(ctypes.byref(net), layer, _p(workspace), ctypes.byref(rows),
                                           ctypes.byref(cap), ctypes.byref(n_rows)), "npvs_forward_layer_output")
    base = workspace.data_ptr()
    return rows.value - base, cap.value, n_rows.value - base


# ---- training: ground truth and a8-a11 ----------------------------------------------------------

def npvs_gt_raycast(boxes, box_offsets, cams_dev, points, g: L.Grid, s_gt: int, gt_bits, g_bits=None,
                    stream=None):
    _need_cuda(boxes, box_offsets, cams_dev, points, gt_bits, g_bits)
    check(_lib().npvs_gt_raycast(_p(boxes), _p(box_offsets), _p(cams_dev), _p(points), points.shape[-2], g, s_gt,
                                 _p(g_bits), _p(gt_bits), _s(stream)), "npvs_gt_raycast")



def npvs_conv_bwd_workspace_bytes(desc: L.ConvDesc) -> int:
    return int(_lib().npvs_conv_bwd_workspace_bytes(ctypes.byref(desc)))


def npvs_sparse_conv_bwd(desc: L.ConvDesc, x, w, y, dy, dx, dx_add, dw, db, workspace, stream=None):
    _need_cuda(x, w, y, dy, dx, dx_add, dw, db, workspace)
    T = _TDT[desc.dtype]
    A = torch.float64 if desc.dtype == L.F64 else torch.float32
    _want(T, x=x, y=y, dy=dy, dx=dx, dx_add=dx_add)
    _want(A, w=w, dw=dw, db=db)
    check(_lib().npvs_sparse_conv_bwd(ctypes.byref(desc), _p(x), _p(w), _p(y), _p(dy), _p(dx), _p(dx_add),
                                      _p(dw), _p(db), _p(workspace), workspace.numel() * workspace.element_size(),
                                      _s(stream)), "npvs_sparse_conv_bwd")


def loss_params(alpha=0.9, eps=1.0, lam=0.99, w_bce=0.0) -> L.LossParams:
    return L.LossParams(alpha, eps, lam, w_bce)


def npvs_loss_workspace_bytes(capacity: int, dtype: int) -> int:
    return int(_lib().npvs_loss_workspace_bytes(capacity, dtype))


def npvs_loss_fwd(dtype: int, logits, coords, n_rows, capacity: int, gt_bits, g_bits, g: L.Grid, d: int,
                  prm: L.LossParams, terms, loss, workspace, stream=None):
    _need_cuda(logits, coords, n_rows, gt_bits, g_bits, terms, loss, workspace)
    _want(_TDT[dtype], logits=logits, terms=terms, loss=loss)
    check(_lib().npvs_loss_fwd(dtype, _p(logits), _p(coords), _p(n_rows), capacity, _p(gt_bits), _p(g_bits), g, d,
                               ctypes.byref(prm), _p(terms), _p(loss), _p(workspace),
                               workspace.numel() * workspace.element_size(), _s(stream)), "npvs_loss_fwd")


def npvs_loss_bwd(dtype: int, logits, coords, n_rows, capacity: int, gt_bits, g_bits, g: L.Grid, d: int,
                  prm: L.LossParams, terms, dloss, dlogits_dtype: int, dlogits, stream=None):
    _need_cuda(logits, coords, n_rows, gt_bits, g_bits, terms, dloss, dlogits)
    _want(_TDT[dtype], logits=logits, terms=terms, dloss=dloss)
    _want(_TDT[dlogits_dtype], dlogits=dlogits)
    check(_lib().npvs_loss_bwd(dtype, _p(logits), _p(coords), _p(n_rows), capacity, _p(gt_bits), _p(g_bits), g, d,
                               ctypes.byref(prm), _p(terms), _p(dloss), dlogits_dtype, _p(dlogits), _s(stream)),
          "npvs_loss_bwd")


def adam_params(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-10) -> L.AdamParams:
    return L.AdamParams(lr, beta1, beta2, eps, weight_decay)


def npvs_adam_step(theta, grad, m, v, prm: L.AdamParams, state, stream=None):
    _need_cuda(theta, grad, m, v, state)
    _want(torch.float32, theta=theta, grad=grad, m=m, v=v)
    _want(torch.int32, state=state)
    check(_lib().npvs_adam_step(_p(theta), _p(grad), _p(m), _p(v), theta.numel(), ctypes.byref(prm), _p(state),
                                _s(stream)), "npvs_adam_step")
