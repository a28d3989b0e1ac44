"""Training of the NeuralPVS network on one GPU through the npvs C ABI (Sec. 3.3, Sec. 4.2).

One step: froxelize the batch's viewcells, interleave, build the rulebooks, run the network
keeping every layer's output, evaluate the weighted Dice + repulsive visibility loss, run the
hand-written backward of the loss and of every convolution in reverse order, take an Adam step
on the FP32 master parameters and repack the BF16 tensor-core weights. Every step is a kernel of
libnpvs.so on the current stream, with all buffers fixed, so the whole step is captured and
replayed as one CUDA graph (`Trainer.capture`).

Precision: BF16 weights and activations on the tensor cores with FP32 accumulation, FP32 logits,
loss, reductions and master weights (dtype BF16); the same in FP32 throughout (dtype F32); FP64
throughout (dtype F64, used by the finite-difference gradient check).

The decoder's up-convolutions add the encoder's output after their ReLU (skip by addition). The
backward needs the ReLU mask of the up-conv's own output, which is not stored: it is recomputed
by running the up-conv again without the skip (activation recomputation of a cheap layer). The
gradient reaching an encoder output through the skip is added by the dgrad of the down-conv that
reads the same output (npvs_sparse_conv_bwd's dx_add), so no separate accumulation runs.

`SparseConv` and `RVLoss` wrap the same entry points as torch.autograd.Functions for callers that
build their own models.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

import torch

from . import _lib as L
from . import ops
from .pipeline import DOWN_KINDS, KIND, TORCH_DT, UP_KINDS, FramePipeline, Net

ALIGN = 64  # elements between parameter tensors in the flat buffers


class Params:
    """Flat master parameters: per layer W [taps][cin][cout] then b [cout], each starting at a
    multiple of ALIGN elements; `grad`, `m`, `v` share the layout (gaps stay zero)."""

    def __init__(self, layers, weights: Sequence, biases: Sequence, dtype=torch.float32, device="cuda"):
        self.layers = list(layers)
        offs, o = [], 0
        for l in self.layers:
            nw = l.taps * l.cin * l.cout
            ow = o
            o = (o + nw + ALIGN - 1) // ALIGN * ALIGN
            ob = o
            o = (o + l.cout + ALIGN - 1) // ALIGN * ALIGN
            offs.append((ow, nw, ob))
        self.n = o
        self.offsets = offs
        self.theta = torch.zeros(o, dtype=dtype, device=device)
        self.grad = torch.zeros_like(self.theta)
        self.w = self._views(self.theta)
        self.b = self._bviews(self.theta)
        self.gw = self._views(self.grad)
        self.gb = self._bviews(self.grad)
        for i in range(len(self.layers)):
            self.w[i].copy_(torch.as_tensor(weights[i]).to(dtype))
            self.b[i].copy_(torch.as_tensor(biases[i]).to(dtype))

    def _views(self, buf):
        return [buf[ow:ow + nw].view(l.taps, l.cin, l.cout) for l, (ow, nw, _) in zip(self.layers, self.offsets)]

    def _bviews(self, buf):
        return [buf[ob:ob + l.cout] for l, (_, _, ob) in zip(self.layers, self.offsets)]


CHECKPOINT_FORMAT = "npvs-trainer-1"


def _layer_key(layers):
    return [(l.name, l.kind, int(l.cin), int(l.cout), bool(l.relu)) for l in layers]


def trainer_state(tr) -> dict:
    """Checkpoint of a Trainer as host tensors (for torch.save): the layer list and dtype (checked
    on load), the master parameters, Adam's moments and its device counters, and the forward's
    tuned kernel forms. With the data sampler's state kept by the caller, a resumed run repeats
    the uninterrupted one bit for bit (every step is deterministic)."""
    return {"format": CHECKPOINT_FORMAT, "layers": _layer_key(tr.layers), "dtype": int(tr.dtype),
            "theta": tr.params.theta.detach().cpu().clone(), "m": tr.m.detach().cpu().clone(),
            "v": tr.v.detach().cpu().clone(), "adam_state": tr.adam_state.detach().cpu().clone(),
            "tuned": tr.pipe.tuned_configs()}


def load_trainer_state(tr, sd: dict):
    """Restores trainer_state() into `tr` in place (every buffer keeps its address, so a graph of
    tr captured earlier replays with the restored parameters; capture again if the tuned forms
    differ) and rebuilds the BF16 weight images. Raises ValueError for another network or dtype."""
    if sd.get("format") != CHECKPOINT_FORMAT:
        raise ValueError(f"not a trainer checkpoint ({sd.get('format')!r})")
    if [tuple(x) for x in sd["layers"]] != _layer_key(tr.layers) or int(sd["dtype"]) != int(tr.dtype):
        raise ValueError("checkpoint of another network or dtype")
    for name, dst in (("theta", tr.params.theta), ("m", tr.m), ("v", tr.v), ("adam_state", tr.adam_state)):
        src = sd[name]
        if tuple(src.shape) != tuple(dst.shape) or src.dtype != dst.dtype:
            raise ValueError(f"checkpoint tensor {name}: {tuple(src.shape)} {src.dtype}, "
                             f"expected {tuple(dst.shape)} {dst.dtype}")
        dst.copy_(src)
    tr.pipe.apply_tuned(sd["tuned"])
    if tr.dtype == L.BF16:
        tr.repack()


class Trainer:
    """Buffers and launch sequence of one training step of `layers` on batches of `batch`
    viewcells of workload `wl`."""

    def __init__(self, wl, layers, weights, biases, batch: int, dtype: int = L.BF16,
                 loss_prm: Optional[L.LossParams] = None, adam_prm: Optional[L.AdamParams] = None,
                 device="cuda", capacity_frac: float = 1.0):
        self.wl, self.B, self.dtype, self.device = wl, batch, dtype, device
        self.layers = list(layers)
        mdt = torch.float64 if dtype == L.F64 else torch.float32
        self.params = Params(layers, weights, biases, mdt, device)
        net = Net.__new__(Net)
        net.layers, net.w32, net.b32, net.device = self.layers, self.params.w, self.params.b, device
        net._packed, net._w64, net._b64 = None, None, None
        self.net = net
        self.pipe = FramePipeline(wl, net, batch, dtype, device=device, capacity_frac=capacity_frac)
        p = self.pipe
        self.loss_prm = loss_prm if loss_prm is not None else ops.loss_params()
        self.adam_prm = adam_prm if adam_prm is not None else ops.adam_params()
        self.gt = torch.zeros_like(p.occ)
        act_dt = TORCH_DT[dtype]
        self.dacts: Dict[str, torch.Tensor] = {l.name: torch.zeros(p.acts[l.name].shape, dtype=act_dt, device=device)
                                               for l in self.layers}
        self.u: Dict[int, torch.Tensor] = {i: torch.zeros_like(p.acts[l.name]) for i, l in enumerate(self.layers)
                                           if l.kind in UP_KINDS}
        self.skip_grad: Dict[int, str] = {}     # down-conv index -> name of the up-conv whose skip it feeds
        lv_of = p._level_of_layers()
        for i, l in enumerate(self.layers):
            if l.kind in DOWN_KINDS:
                self.skip_grad[i] = next((m.name for m in self.layers
                                          if m.kind in UP_KINDS and lv_of[m.name] == lv_of[l.name] - 1), None)
        self.bwd_ws = ops.conv_workspace(max(ops.npvs_conv_bwd_workspace_bytes(d) for d in p.descs), device)
        self.loss_dtype = L.F64 if dtype == L.F64 else L.F32
        ldt = TORCH_DT[self.loss_dtype]
        self.terms = torch.zeros(batch, L.LOSS_TERMS, dtype=ldt, device=device)
        self.loss = torch.zeros(1, dtype=ldt, device=device)
        self.loss_ws = ops.conv_workspace(ops.npvs_loss_workspace_bytes(p.levels[0].capacity, self.loss_dtype),
                                          device)
        self.m = torch.zeros_like(self.params.theta)
        self.v = torch.zeros_like(self.params.theta)
        self.adam_state = torch.zeros(2, dtype=torch.int32, device=device)
        self.packed: List[torch.Tensor] = []
        self.packed_t: List[Optional[torch.Tensor]] = []   # dgrad images (BF16 tensor-core layers)
        if dtype == L.BF16:
            jobs = []
            for i, l in enumerate(self.layers):
                k = KIND[l.kind]
                self.packed.append(torch.empty(ops.npvs_packed_weight_bytes(k, l.cin, l.cout),
                                               dtype=torch.uint8, device=device))
                jobs.append((k, l.cin, l.cout, 0, self.params.w[i], self.packed[i]))
                # the first layer's input has no gradient: no dgrad image
                nt = ops.npvs_packed_weight_bytes_transposed(k, l.cin, l.cout) if i > 0 else 0
                self.packed_t.append(torch.empty(nt, dtype=torch.uint8, device=device) if nt else None)
                if nt:
                    jobs.append((k, l.cin, l.cout, 1, self.params.w[i], self.packed_t[i]))
            self._pack_jobs = ops.make_pack_jobs(jobs)
            self.repack()

    def state_dict(self) -> dict:
        return trainer_state(self)

    def load_state_dict(self, sd: dict):
        load_trainer_state(self, sd)

    def autotune(self, boxes, box_offsets, cams_dev, reps: int = 3):
        """Per-layer kernel configurations of the forward convolutions, timed on this batch (see
        FramePipeline.autotune); the backward keeps its defaults. Returns {layer: (config, us)}."""
        return self.pipe.autotune(boxes, box_offsets, cams_dev, reps=reps)

    # ---- parts of a step ----------------------------------------------------------------------
    def repack(self):
        """BF16 tensor-core images of the current master weights: every layer's forward image and
        the image its backward's dgrad reads, in one launch per 24 layers."""
        ops.npvs_pack_weights_many(self._pack_jobs)

    def _operands(self):
        return self.packed if self.dtype == L.BF16 else self.params.w

    def _input_of(self, i):
        return self.pipe.feats if i == 0 else self.pipe.acts[self.layers[i - 1].name]

    def forward(self, boxes, box_offsets, cams_dev):
        p = self.pipe
        p.froxelize(boxes, box_offsets, cams_dev)
        p.interleave()
        p.rulebooks()
        self.network()

    def network(self):
        p, W = self.pipe, self._operands()
        for i, l in enumerate(self.layers):
            ops.npvs_sparse_conv_fwd(p.descs[i], self._input_of(i), W[i], self.params.b[i], p.skip_of.get(i),
                                     p.acts[l.name])

    def loss_forward(self):
        p = self.pipe
        lv0 = p.levels[0]
        ops.npvs_loss_fwd(self.loss_dtype, p.logits, lv0.coords, lv0.n_rows, lv0.capacity, self.gt, p.occ, p.grid,
                          self.wl.d, self.loss_prm, self.terms, self.loss, self.loss_ws)

    def backward(self):
        p, W = self.pipe, self._operands()
        lv0 = p.levels[0]
        head = self.layers[-1].name
        ops.npvs_loss_bwd(self.loss_dtype, p.logits, lv0.coords, lv0.n_rows, lv0.capacity, self.gt, p.occ, p.grid,
                          self.wl.d, self.loss_prm, self.terms, None, self.dtype, self.dacts[head])
        for i in range(len(self.layers) - 1, -1, -1):
            l = self.layers[i]
            desc = p.descs[i]
            x = self._input_of(i)
            y = p.acts[l.name]
            if l.kind in UP_KINDS:   # recompute the up-conv's own output (before the skip) for its ReLU mask
                ops.npvs_sparse_conv_fwd(desc, x, W[i], self.params.b[i], None, self.u[i])
                y = self.u[i]
            dx = None if i == 0 else self.dacts[self.layers[i - 1].name]
            sg = self.skip_grad.get(i)
            wt = self.packed_t[i] if self.dtype == L.BF16 and dx is not None else None
            desc.w_transposed = wt.data_ptr() if wt is not None else None
            try:
                ops.npvs_sparse_conv_bwd(desc, x, self.params.w[i], y if l.relu else None, self.dacts[l.name], dx,
                                         self.dacts[sg] if sg else None, self.params.gw[i], self.params.gb[i],
                                         self.bwd_ws)
            finally:
                desc.w_transposed = None

    def optimizer_step(self):
        ops.npvs_adam_step(self.params.theta, self.params.grad, self.m, self.v, self.adam_prm, self.adam_state)
        if self.dtype == L.BF16:
            self.repack()

    def step(self, boxes, box_offsets, cams_dev, update: bool = True):
        self.forward(boxes, box_offsets, cams_dev)
        self.loss_forward()
        self.backward()
        if update:
            self.optimizer_step()

    def capture(self, boxes, box_offsets, cams_dev, update: bool = True):
        """One training step as a CUDA graph over fixed input buffers (boxes, box_offsets,
        cams_dev, self.gt). The warm-up step runs outside the capture and does update the
        parameters when `update` is set."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.step(boxes, box_offsets, cams_dev, update)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step(boxes, box_offsets, cams_dev, update)
        return g


# ---- autograd wrappers ---------------------------------------------------------------------------

class SparseConv(torch.autograd.Function):
    """y = relu?(conv(x) + b) (+ skip) with the npvs kernels. `desc` is the layer's forward
    descriptor (maps and row counts of a built level pair); `operand` the weight operand the
    forward reads (the packed image for BF16, else w itself); w and b are the master parameters.
    Output rows past the level's row count are zero."""

    @staticmethod
    def forward(ctx, x, w, b, skip, desc, operand, cout_rows: int, y_dtype):
        y = torch.zeros(cout_rows, desc.cout, dtype=y_dtype, device=x.device)
        ops.npvs_sparse_conv_fwd(desc, x, operand, b, skip, y)
        ctx.desc, ctx.operand, ctx.has_skip = desc, operand, skip is not None
        if skip is None:
            ctx.save_for_backward(x, w, b, y)
        else:
            ctx.save_for_backward(x, w, b)
        return y

    @staticmethod
    def backward(ctx, dy):
        x, w, b = ctx.saved_tensors[:3]
        d = L.ConvDesc.from_buffer_copy(ctx.desc)
        d.w_transposed = None            # the dgrad image is packed from w in the call
        y = None
        if d.relu:
            if ctx.has_skip:   # recompute the output before the skip for the ReLU mask
                y = torch.zeros(dy.shape[0], d.cout, dtype=dy.dtype, device=dy.device)
                ops.npvs_sparse_conv_fwd(d, x, ctx.operand, b, None, y)
            else:
                y = ctx.saved_tensors[3]
        dy = dy.contiguous()
        dx = torch.zeros_like(x) if ctx.needs_input_grad[0] else None
        dw = torch.zeros_like(w)
        db = torch.zeros_like(b)
        ws = ops.conv_workspace(ops.npvs_conv_bwd_workspace_bytes(d), dy.device)
        ops.npvs_sparse_conv_bwd(d, x, w, y, dy, dx, None, dw, db, ws)
        return dx, dw, db, (dy if ctx.has_skip else None), None, None, None, None


class RVLoss(torch.autograd.Function):
    """Weighted Dice + repulsive visibility loss (Sec. 3.3) of the logits of one interleaved
    level against ground-truth and geometry bit grids; returns the batch mean (shape [1])."""

    @staticmethod
    def forward(ctx, logits, coords, n_rows, gt_bits, g_bits, grid: L.Grid, d: int, prm: L.LossParams,
                dlogits_dtype: int):
        dt = L.F64 if logits.dtype == torch.float64 else L.F32
        B = grid.B
        terms = torch.zeros(B, L.LOSS_TERMS, dtype=logits.dtype, device=logits.device)
        loss = torch.zeros(1, dtype=logits.dtype, device=logits.device)
        ws = ops.conv_workspace(ops.npvs_loss_workspace_bytes(logits.shape[0], dt), logits.device)
        ops.npvs_loss_fwd(dt, logits, coords, n_rows, logits.shape[0], gt_bits, g_bits, grid, d, prm, terms, loss, ws)
        ctx.save_for_backward(logits, coords, n_rows, gt_bits, g_bits, terms)
        ctx.grid, ctx.d, ctx.prm, ctx.dt, ctx.odt = grid, d, prm, dt, dlogits_dtype
        ctx.mark_non_differentiable(terms)
        return loss, terms

    @staticmethod
    def backward(ctx, dloss, dterms):
        logits, coords, n_rows, gt_bits, g_bits, terms = ctx.saved_tensors
        out = torch.zeros(logits.shape, dtype=TORCH_DT[ctx.odt], device=logits.device)
        ops.npvs_loss_bwd(ctx.dt, logits, coords, n_rows, logits.shape[0], gt_bits, g_bits, ctx.grid, ctx.d, ctx.prm,
                          terms, dloss.contiguous().to(logits.dtype), ctx.odt, out)
        return out, None, None, None, None, None, None, None, None
