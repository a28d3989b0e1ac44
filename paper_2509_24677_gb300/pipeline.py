"""Per-frame NeuralPVS inference on one GPU through the npvs C ABI.

V = g_d^-1(f_theta(g_d(G))) thresholded at tau and masked by G (Sec. 3.1-3.3), with G the
froxelized scene of the viewcell's enclosing frustum (Sec. 3.2). All device buffers are
allocated once per (workload, batch, dtype) with capacity-bounded sizes; every step is a kernel
of libnpvs.so enqueued on the current stream, with row counts kept on the device, so a frame can
be replayed as a CUDA graph.
"""
from __future__ import annotations

import contextlib
import dataclasses
from typing import Dict, List, Optional, Sequence

import torch

from . import _lib as L
from . import ops

TORCH_DT = {L.F32: torch.float32, L.BF16: torch.bfloat16, L.F64: torch.float64}
DOWN_KINDS = ("down2", "down3")
UP_KINDS = ("up2", "up3")
KIND = {"subm3": L.CONV_SUBM3, "down2": L.CONV_DOWN2, "up2": L.CONV_UP2, "head1": L.CONV_HEAD1,
        "down3": L.CONV_DOWN3, "up3": L.CONV_UP3}


@dataclasses.dataclass
class SparseLevel:
    dims: L.Dims
    capacity: int
    coords: torch.Tensor     # [cap][4] int32
    n_rows: torch.Tensor     # [1] int32
    table: torch.Tensor      # [B*Z*Y*X] int32
    nbr: torch.Tensor        # [cap][27] int32
    down: Optional[torch.Tensor] = None   # [cap_next][8] child rows of each parent (next level)
    up: Optional[torch.Tensor] = None     # [cap][1] parent*8 + tap

    @staticmethod
    def alloc(X, Y, Z, B, cap, device):
        n_sites = X * Y * Z * B
        i32 = dict(dtype=torch.int32, device=device)
        return SparseLevel(L.Dims(X, Y, Z, B), cap, torch.zeros(cap, 4, **i32), torch.zeros(1, **i32),
                           torch.empty(n_sites, **i32), torch.empty(cap, 27, **i32))


def _timing_event():
    # "external" events stay queryable when recorded inside a CUDA graph capture
    try:
        return torch.cuda.Event(enable_timing=True, external=True)
    except TypeError:
        return torch.cuda.Event(enable_timing=True)


class StageTimer:
    """Records a CUDA event pair around each named stage on the current stream."""

    def __init__(self):
        self.events = []

    @contextlib.contextmanager
    def __call__(self, name):
        s = _timing_event()
        e = _timing_event()
        s.record()
        yield
        e.record()
        self.events.append((name, s, e))

    def totals(self) -> Dict[str, float]:
        out: Dict[str, float] = {}
        for name, s, e in self.events:
            out[name] = out.get(name, 0.0) + s.elapsed_time(e)
        return out


_null = contextlib.nullcontext()


class Net:
    """Network weights on the device: FP32 master [taps][cin][cout], biases, and per dtype the
    operand the kernels read (packed BF16 tiles, or the FP32/FP64 tensors themselves)."""

    def __init__(self, layers, weights: Sequence, biases: Sequence, device="cuda"):
        self.layers = list(layers)
        self.w32 = [torch.as_tensor(w, dtype=torch.float32).contiguous().to(device) for w in weights]
        self.b32 = [torch.as_tensor(b, dtype=torch.float32).contiguous().to(device) for b in biases]
        self.device = device
        self._packed: Optional[List[torch.Tensor]] = None
        self._w64: Optional[List[torch.Tensor]] = None

    def packed(self) -> List[torch.Tensor]:
        if self._packed is None:
            self._packed = [torch.empty(ops.npvs_packed_weight_bytes(KIND[l.kind], l.cin, l.cout), dtype=torch.uint8,
                                        device=self.device) for l in self.layers]
            ops.npvs_pack_weights_many([(KIND[l.kind], l.cin, l.cout, 0, w, buf)
                                        for l, w, buf in zip(self.layers, self.w32, self._packed)])
        return self._packed

    def repack(self):
        self._packed = None
        self._w64 = None
        self._b64 = None

    def operands(self, dtype):
        if dtype == L.BF16:
            return self.packed()
        if dtype == L.F64:
            if self._w64 is None:
                self._w64 = [w.double() for w in self.w32]
            return self._w64
        return self.w32

    def biases(self, dtype):
        """Bias operands: FP32, or FP64 copies for the FP64 path."""
        if dtype == L.F64:
            if getattr(self, "_b64", None) is None:
                self._b64 = [b.double() for b in self.b32]
            return self._b64
        return self.b32


def chain_layer_indices(layers, chain_level: int) -> List[int]:
    """Indices of the layers npvs_forward runs as one persistent launch for `chain_level` (0: none):
    the down conv into that level through the up conv out of it."""
    if chain_level <= 0:
        return []
    lv, first = 0, None
    for i, l in enumerate(layers):
        if l.kind in DOWN_KINDS:
            lv += 1
            if first is None and lv == chain_level:
                first = i
        elif l.kind in UP_KINDS:
            lv -= 1
            if first is not None and lv == chain_level - 1:
                return list(range(first, i + 1))
    return []


class FramePipeline:
    """Buffers and launch sequence of one frame (batch of viewcells) for a workload."""

    def __init__(self, wl, net: Net, batch: int = 1, dtype: int = L.BF16, tau: float = 0.5,
                 device="cuda", capacity_frac: float = 1.0):
        self.wl, self.net, self.B, self.dtype, self.tau = wl, net, batch, dtype, tau
        self.device = device
        d = wl.d
        self.grid = L.Grid(wl.W, wl.H, wl.D, batch)
        self.n_levels = 1 + sum(1 for l in net.layers if l.kind in DOWN_KINDS)
        # k = 3 stride-2 pair: each coarser level is the dilated output set of a DOWN3 rulebook
        self.k3 = any(l.kind in ("down3", "up3") for l in net.layers)
        taps = 27 if self.k3 else 8
        i32 = dict(dtype=torch.int32, device=device)
        self.occ = torch.empty(batch * wl.D * wl.H * (wl.W // 32), **i32)
        self.pvs = torch.empty_like(self.occ)
        self.status = torch.zeros(1, **i32)
        self.levels: List[SparseLevel] = []
        X, Y, Z = wl.W // d, wl.H // d, wl.D // d
        for li in range(self.n_levels):
            sites = X * Y * Z * batch
            cap = max(1, int(sites * capacity_frac))
            self.levels.append(SparseLevel.alloc(X, Y, Z, batch, cap, device))
            X, Y, Z = X // 2, Y // 2, Z // 2
        for li in range(self.n_levels - 1):
            a, b = self.levels[li], self.levels[li + 1]
            a.down = torch.empty(b.capacity, taps, **i32)   # input rows of each coarse output
            a.up = torch.empty(a.capacity, 27 if self.k3 else 1, **i32)
        act_dt = TORCH_DT[dtype]
        cap0 = self.levels[0].capacity
        self.feats = torch.zeros(cap0, wl.feat_ch, dtype=act_dt, device=device)
        self.acts: Dict[str, torch.Tensor] = {}
        lv_of = self._level_of_layers()
        last = net.layers[-1].name
        for l in net.layers:
            cap = self.levels[lv_of[l.name]].capacity
            # the last layer's logits are FP32 on every path but FP64
            dt = torch.float32 if (l.name == last and dtype != L.F64) else act_dt
            self.acts[l.name] = torch.zeros(cap, l.cout, dtype=dt, device=device)
        self.logits = self.acts[net.layers[-1].name]
        self.probs = torch.zeros(cap0, d ** 3, dtype=torch.float32, device=device)
        self.ws = ops.Workspace(device)
        self.timer: Optional[StageTimer] = None
        self._build_descs()

    def _t(self, name):
        return self.timer(name) if self.timer is not None else _null

    def _level_of_layers(self):
        lv, out = 0, {}
        for l in self.net.layers:
            if l.kind in DOWN_KINDS:
                lv += 1
            elif l.kind in UP_KINDS:
                lv -= 1
            out[l.name] = lv
        return out

    # ------------------------------------------------------------------------------------------
    def froxelize(self, boxes, box_offsets, cams_dev):
        with self._t("froxelize"):
            ops.npvs_froxelize(boxes, box_offsets, cams_dev, self.grid, self.wl.supersample, self.occ, ws=self.ws)

    def interleave(self):
        lv0 = self.levels[0]
        with self._t("interleave"):
            ops.npvs_interleave(self.occ, self.grid, self.wl.d, self.wl.in_ch, self.dtype, lv0.capacity,
                                lv0.coords, self.feats, lv0.n_rows, table=lv0.table, status=self.status, ws=self.ws)

    def rulebooks(self):
        with self._t("rulebooks"):
            for li, lv in enumerate(self.levels):
                # every level's table is already written (level 0 by the interleave, the others by
                # the down rulebook), so only the neighbour map is built
                ops.npvs_build_rulebook(L.RB_SUBM3_TABLE, lv, None, lv.nbr, status=self.status, ws=self.ws)
                if li + 1 < self.n_levels:
                    nxt = self.levels[li + 1]
                    ops.npvs_build_rulebook(L.RB_DOWN3 if self.k3 else L.RB_DOWN2, lv, nxt, lv.down, lv.up,
                                            status=self.status, ws=self.ws)

    def _build_descs(self):
        """Descriptors of every layer (fixed buffers), the shared convolution workspace sized for the
        largest product-form tile set, and the skip input of each decoder up-conv."""
        lv_of = self._level_of_layers()
        self.descs, self.skip_of = [], {}
        for i, l in enumerate(self.net.layers):
            li = lv_of[l.name]
            lv = self.levels[li]
            last = i == len(self.net.layers) - 1
            common = dict(out_f32=last, status=self.status)
            if l.kind == "subm3":
                d = ops.conv_desc(L.CONV_SUBM3, self.dtype, l.cin, l.cout, l.relu, lv.nbr, lv.n_rows, lv.capacity,
                                  n_in=lv.n_rows, cap_in=lv.capacity, **common)
            elif l.kind in DOWN_KINDS:   # map: the input rows of each output, map2: the level pair's other map
                prev = self.levels[li - 1]
                d = ops.conv_desc(KIND[l.kind], self.dtype, l.cin, l.cout, l.relu, prev.down, lv.n_rows, lv.capacity,
                                  map2=prev.up, n_in=prev.n_rows, cap_in=prev.capacity, **common)
            elif l.kind in UP_KINDS:
                nxt = self.levels[li + 1]
                d = ops.conv_desc(KIND[l.kind], self.dtype, l.cin, l.cout, l.relu, lv.up, lv.n_rows, lv.capacity,
                                  map2=lv.down, n_in=nxt.n_rows, cap_in=nxt.capacity, **common)
                self.skip_of[i] = self.acts[f"enc{li}b"]
            else:
                d = ops.conv_desc(L.CONV_HEAD1, self.dtype, l.cin, l.cout, l.relu, None, lv.n_rows, lv.capacity,
                                  n_in=lv.n_rows, cap_in=lv.capacity, **common)
            self.descs.append(d)
        self.conv_ws = None
        if self.dtype in (L.BF16, L.F32):     # tensor-core / FP32 product tiles and split-K partials
            nbytes = max(ops.npvs_conv_workspace_bytes(d) for d in self.descs)
            self.conv_ws = ops.conv_workspace(nbytes, self.device)
            for d in self.descs:
                d.workspace = self.conv_ws.data_ptr()
                d.workspace_bytes = self.conv_ws.numel()

    def network(self):
        W = self.net.operands(self.dtype)
        Bs = self.net.biases(self.dtype)
        a = self.feats
        for i, l in enumerate(self.net.layers):
            y = self.acts[l.name]
            with self._t("conv:" + l.name):
                ops.npvs_sparse_conv_fwd(self.descs[i], a, W[i], Bs[i], self.skip_of.get(i), y)
            a = y
        return a

    # ---- autotuning ------------------------------------------------------------------------------
    CANDIDATES = {
        "subm3": [dict(tune_form=2), dict(tune_form=2, tune_max_split=8), dict(tune_form=1, tune_gather_warps=8),
                  dict(tune_form=1, tune_gather_warps=8, tune_max_split=1), dict(tune_form=1, tune_gather_warps=4),
                  dict(tune_form=1, tune_gather=3), dict(tune_form=1, tune_gather=3, tune_max_split=1),
                  dict(tune_form=1, tune_gather=3, tune_gather_warps=4), dict(tune_form=1, tune_gather=4),
                  dict(tune_form=1, tune_gather=4, tune_max_split=1)],
        "down2": [dict(tune_form=2), dict(tune_form=2, tune_max_split=8), dict(tune_form=1, tune_gather_warps=8),
                  dict(tune_form=1, tune_gather_warps=8, tune_max_split=1)],
        "up2": [dict(tune_form=2), dict(tune_form=1)],
        "down3": [dict(tune_form=2), dict(tune_form=1), dict(tune_form=1, tune_max_split=1)],
        "up3": [dict(tune_form=2), dict(tune_form=1), dict(tune_form=1, tune_max_split=1)],
        "head1": [dict()],
    }

    def autotune(self, boxes, box_offsets, cams_dev, reps: int = 10, record: Optional[dict] = None,
                 margin: float = 0.05, refine_window: float = 0.15):
        """Times the candidate configurations of every BF16 layer on this frame (each as a CUDA
        graph of `reps` launches) and keeps the fastest in the layer's descriptor. The best choice
        depends on the active-site counts, so tune on a representative frame. A candidate replaces
        an earlier one in CANDIDATES (product form, then gather, then window forms) only when it is
        faster by more than `margin`: timed alone, one layer's launches understate the in-frame
        cost of the one-kernel forms against the two-kernel product form by a few percent (level-1
        layers of the 256x256x128 frame: 24.5 / 23.8 us alone, 30.5 / 27.3 us in the frame).
        Then every layer whose runner-up (another form) is within `refine_window` of its best is
        decided in the frame: the frame is captured with the stage timer once with the winners and
        once with the runners-up, and per layer the form with the shorter in-frame time is kept.
        Returns {layer: (config, microseconds)}; `record`, if given, receives every candidate's
        time as {layer: [(config, microseconds), ...]}."""
        if self.dtype != L.BF16:
            return {}
        self.run(boxes, box_offsets, cams_dev, want_probs=False)
        torch.cuda.synchronize()
        W = self.net.operands(self.dtype)
        chosen = {}
        times: Dict[int, list] = {}
        x = self.feats
        for i, l in enumerate(self.net.layers):
            y = self.acts[l.name]
            best = None
            for cfg in self.CANDIDATES[l.kind]:
                d = L.ConvDesc.from_buffer_copy(self.descs[i])
                for k, v in cfg.items():
                    setattr(d, k, v)
                args = (d, x, W[i], self.net.b32[i], self.skip_of.get(i), y)
                ops.npvs_sparse_conv_fwd(*args)
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    for _ in range(reps):
                        ops.npvs_sparse_conv_fwd(*args)
                g.replay()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                g.replay()
                e1.record()
                torch.cuda.synchronize()
                us = e0.elapsed_time(e1) * 1000.0 / reps
                times.setdefault(i, []).append((cfg, us))
                if record is not None:
                    record.setdefault(l.name, []).append((cfg, us))
                if best is None or us < best[1] * (1.0 - margin):
                    best = (cfg, us)
            self._apply_cfg(i, best[0])
            chosen[l.name] = best
            x = y
        # close calls are decided in the frame
        alt = {}
        for i, l in enumerate(self.net.layers):
            cfg, us = chosen[l.name]
            runners = sorted((c for c in times[i] if c[0] != cfg), key=lambda c: c[1])
            if runners and runners[0][1] <= us * (1.0 + refine_window):
                alt[i] = runners[0]
        if alt:
            t_best = self._frame_layer_times(boxes, box_offsets, cams_dev)
            for i, (cfg, _) in alt.items():
                self._apply_cfg(i, cfg)
            t_alt = self._frame_layer_times(boxes, box_offsets, cams_dev)
            for i, (cfg, us) in alt.items():
                name = self.net.layers[i].name
                if t_alt[name] < t_best[name]:
                    chosen[name] = (cfg, us)
                else:
                    self._apply_cfg(i, chosen[name][0])
        self.run(boxes, box_offsets, cams_dev, want_probs=False)   # outputs with the chosen configs
        torch.cuda.synchronize()
        return chosen

    def use_chain_forms(self, chain_level: int):
        """Runs the layers that npvs_forward chains at `chain_level` in the product form, the form
        the chain computes, so that this frame and NativeFrame(chain_level=...) agree bit for bit."""
        for i in chain_layer_indices(self.net.layers, chain_level):
            self._apply_cfg(i, dict(tune_form=2))

    def _apply_cfg(self, i: int, cfg: dict):
        for f in self.TUNE_FIELDS:
            setattr(self.descs[i], f, int(cfg.get(f, 0)))

    def _frame_layer_times(self, boxes, box_offsets, cams_dev, replays: int = 6) -> Dict[str, float]:
        """Per-layer times (ms) inside a stage-timed graph of this frame with the current configs."""
        timer = StageTimer()
        g = self.capture(boxes, box_offsets, cams_dev, want_probs=False, timer=timer)
        acc: Dict[str, float] = {}
        for r in range(replays):
            g.replay()
            torch.cuda.synchronize()
            if r >= 1:
                for k, v in timer.totals().items():
                    if k.startswith("conv:"):
                        acc[k[5:]] = acc.get(k[5:], 0.0) + v
        del g
        return acc

    TUNE_FIELDS = ("tune_stages", "tune_max_split", "tune_lag", "tune_gather", "tune_gather_warps", "tune_form")

    def tuned_configs(self) -> dict:
        """The per-layer kernel configurations in use: {layer name: {field: value}}."""
        return {l.name: {f: int(getattr(self.descs[i], f)) for f in self.TUNE_FIELDS}
                for i, l in enumerate(self.net.layers)}

    def apply_tuned(self, cfgs: dict):
        """Sets per-layer kernel configurations saved by tuned_configs() (instead of autotune)."""
        for i, l in enumerate(self.net.layers):
            for f, v in cfgs[l.name].items():
                setattr(self.descs[i], f, int(v))

    def deinterleave(self, want_probs=True):
        lv0 = self.levels[0]
        with self._t("deinterleave"):
            ops.npvs_deinterleave(self.logits, lv0.table, lv0.n_rows, self.grid, self.wl.d, self.tau, self.occ,
                                  self.pvs, probs_out=self.probs if want_probs else None, capacity=lv0.capacity)

    def run(self, boxes, box_offsets, cams_dev, want_probs=True):
        self.froxelize(boxes, box_offsets, cams_dev)
        self.interleave()
        self.rulebooks()
        self.network()
        self.deinterleave(want_probs)

    # ---- CUDA graph of one frame ------------------------------------------------------------
    def capture(self, boxes, box_offsets, cams_dev, want_probs=False, timer: Optional[StageTimer] = None):
        """Captures one frame into a CUDA graph over fixed input buffers (boxes, box_offsets,
        cams_dev); refill those buffers and call graph.replay() per frame. With `timer`, the stage
        events are captured too and hold the stage times of the latest replay."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.run(boxes, box_offsets, cams_dev, want_probs)   # warm-up outside capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        self.timer = timer
        try:
            with torch.cuda.graph(g):
                self.run(boxes, box_offsets, cams_dev, want_probs)
        finally:
            self.timer = None
        return g

    def frame_from_host(self, graph, cam_buf, cam_host, pvs_host):
        """One frame through a captured graph with host buffers: upload the camera (pinned host
        npvs_camera bytes), replay, download the PVS bits into pinned host memory (async)."""
        cam_buf.copy_(cam_host, non_blocking=True)
        graph.replay()
        pvs_host.copy_(self.pvs, non_blocking=True)


class NativeFrame:
    """A frame through the single native call npvs_forward: the same kernels in the same order as
    FramePipeline, with every buffer carved from one caller-owned workspace. `tuned` (a
    FramePipeline's descriptors) copies per-layer kernel configurations chosen by its autotuner."""

    def __init__(self, wl, net: Net, batch: int = 1, dtype: int = L.BF16, tau: float = 0.5, max_boxes: int = 4096,
                 device="cuda", capacity_frac: float = 1.0, tuned: Optional[Sequence[L.ConvDesc]] = None,
                 chain_level: int = 0):
        self.wl, self.net, self.B, self.dtype = wl, net, batch, dtype
        self.chain_level = chain_level
        W = net.operands(dtype)
        Bs = net.biases(dtype)
        self._keep = (W, Bs)
        n = len(net.layers)
        self.layers_c = (L.NetLayer * n)()
        for i, l in enumerate(net.layers):
            c = self.layers_c[i]
            c.kind, c.cin, c.cout, c.relu = KIND[l.kind], l.cin, l.cout, int(l.relu)
            c.w, c.bias = W[i].data_ptr(), Bs[i].data_ptr()
            if tuned is not None:
                for f in ("tune_stages", "tune_max_split", "tune_lag", "tune_gather", "tune_gather_warps", "tune_form"):
                    setattr(c, f, getattr(tuned[i], f))
        permille = 0 if capacity_frac >= 1.0 else max(1, int(round(capacity_frac * 1000)))
        self.grid = L.Grid(wl.W, wl.H, wl.D, batch)
        self.desc = L.NetDesc(self.grid, wl.d, wl.in_ch, wl.supersample, dtype, tau, max_boxes, permille, n,
                              self.layers_c, chain_level)
        nbytes = ops.npvs_forward_workspace_bytes(self.desc)
        if nbytes == 0:
            raise ValueError("npvs_forward: invalid network plan")
        self.ws = torch.zeros(nbytes, dtype=torch.uint8, device=device)
        i32 = dict(dtype=torch.int32, device=device)
        self.occ = torch.zeros(batch * wl.D * wl.H * (wl.W // 32), **i32)
        self.pvs = torch.zeros_like(self.occ)
        self.status = torch.zeros(1, **i32)
        off, cap, _ = ops.npvs_forward_layer_output(self.desc, -1, self.ws)
        self.probs = torch.zeros(cap, wl.d ** 3, dtype=torch.float32, device=device)

    def layer_output(self, i: int):
        """(rows [capacity][C] view into the workspace, row-count tensor view) of layer i (-1: the
        interleaved input)."""
        off, cap, noff = ops.npvs_forward_layer_output(self.desc, i, self.ws)
        if i < 0:
            C, dt = self.wl.feat_ch, TORCH_DT[self.dtype]
        else:
            C = self.net.layers[i].cout
            dt = torch.float32 if i == len(self.net.layers) - 1 else TORCH_DT[self.dtype]
        nb = cap * C * torch.empty(0, dtype=dt).element_size()
        rows = self.ws[off:off + nb].view(dt).view(cap, C)
        return rows, self.ws[noff:noff + 4].view(torch.int32)

    def run(self, boxes, box_offsets, n_boxes: int, cams_dev, want_probs: bool = False):
        ops.npvs_forward(self.desc, boxes, box_offsets, n_boxes, cams_dev, self.occ, self.pvs,
                         self.probs if want_probs else None, self.status, self.ws)

    def capture(self, boxes, box_offsets, n_boxes: int, cams_dev, want_probs: bool = False):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.run(boxes, box_offsets, n_boxes, cams_dev, want_probs)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(boxes, box_offsets, n_boxes, cams_dev, want_probs)
        return g

    def frame_from_host(self, graph, cam_buf, cam_host, pvs_host):
        cam_buf.copy_(cam_host, non_blocking=True)
        graph.replay()
        pvs_host.copy_(self.pvs, non_blocking=True)
