"""Oracle sparse convolutions and networks in FP64 (test infrastructure; see ``oracle/__init__``).

Sec. 2.3: sparse convolution stores only active sites (hash-indexed); the submanifold variant
(Graham) keeps the output set equal to the input set by centring the kernel on active sites;
strided/transposed variants change resolution. Sec. 3.3: the network f_theta maps the
interleaved grid to per-froxel probabilities.

Each layer is written as the plain dense definition evaluated on the zero-filled grid, at the
active output sites only, which is what the sparse variants compute:
  SubM3     y[p] = b + sum_{delta in {-1,0,1}^3} W_delta^T x[p + delta]         (output set = input set)
            tap k = ((dz+1)*3 + (dy+1))*3 + (dx+1)
  down2     y[P] = b + sum_{c in {0,1}^3} W_c^T x[2P + c]                      (output set = {floor(p/2)})
            tap j = (cz*2 + cy)*2 + cx
  up2       transposed stride-2 conv: out[2P + c] = b + W_c^T z[P], read at the finer level's
            active set (the encoder set of that level)
  head1     y[p] = b + W_0^T x[p]
  down3     k = 3, stride 2, padding 1: y[q] = b + sum_{k in {0,1,2}^3} W_k^T x[2q + k - 1] at the
            dilated output set {q : some 2q + k - 1 active}; tap (kz*3 + ky)*3 + kx
  up3       its transpose: out[2q + k - 1] += W_k^T z[q], read at the finer level's active set
Inactive inputs are zero, which is the "masked dense convolution" reading.

Readings (the workloads name channel widths only): ReLU after every layer except the head;
U-Net: stem SubM3, per level two SubM3 then down2, decoder per level up2 then addition of the
encoder level's output (skip), then two SubM3; head 1x1 to d^3 logits; no normalisation.
Gradients are those of these definitions, computed by torch autograd in float64.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np
import torch

OFFS27 = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
K27 = [(kz, ky, kx) for kz in range(3) for ky in range(3) for kx in range(3)]
CHILD8 = [(cz, cy, cx) for cz in (0, 1) for cy in (0, 1) for cx in (0, 1)]

F64 = torch.float64


class Level:
    """Active sites of one resolution: coords [N][4] (b, z, y, x) in linear order, grid dims."""

    def __init__(self, coords, dims: Tuple[int, int, int, int]):
        self.coords = torch.as_tensor(np.asarray(coords), dtype=torch.long).reshape(-1, 4)
        self.dims = tuple(int(v) for v in dims)   # (B, Dz, Hy, Wx)

    @property
    def n(self) -> int:
        return int(self.coords.shape[0])

    def parent(self) -> "Level":
        B, Dz, Hy, Wx = self.dims
        assert Dz % 2 == 0 and Hy % 2 == 0 and Wx % 2 == 0
        c = self.coords.clone()
        c[:, 1:] //= 2
        pd = (B, Dz // 2, Hy // 2, Wx // 2)
        lin = ((c[:, 0] * pd[1] + c[:, 1]) * pd[2] + c[:, 2]) * pd[3] + c[:, 3]
        u = torch.unique(lin)          # sorted = linear order
        Wp, Hp, Dp = pd[3], pd[2], pd[1]
        pc = torch.stack([u // (Dp * Hp * Wp), (u // (Hp * Wp)) % Dp, (u // Wp) % Hp, u % Wp], 1)
        return Level(pc, pd)

    def strided3(self) -> "Level":
        """The output set of a k = 3, stride 2, padding 1 convolution: the halved-grid sites whose
        3^3 input window {2q - 1, 2q, 2q + 1}^3 holds an active site (max-pooling of the indicator)."""
        B, Dz, Hy, Wx = self.dims
        assert Dz % 2 == 0 and Hy % 2 == 0 and Wx % 2 == 0
        ind = torch.zeros((B, 1, Dz, Hy, Wx), dtype=F64)
        c = self.coords
        ind[c[:, 0], 0, c[:, 1], c[:, 2], c[:, 3]] = 1.0
        pooled = torch.nn.functional.max_pool3d(ind, kernel_size=3, stride=2, padding=1)[:, 0]
        assert pooled.shape[1:] == (Dz // 2, Hy // 2, Wx // 2)
        return Level(torch.nonzero(pooled > 0), (B, Dz // 2, Hy // 2, Wx // 2))


def _dense(level: Level, x: torch.Tensor, halo: int) -> torch.Tensor:
    B, Dz, Hy, Wx = level.dims
    g = torch.zeros((B, Dz + 2 * halo, Hy + 2 * halo, Wx + 2 * halo, x.shape[1]), dtype=x.dtype)
    c = level.coords
    return g.index_put((c[:, 0], c[:, 1] + halo, c[:, 2] + halo, c[:, 3] + halo), x)


def subm3(level: Level, x, W, b):
    g = _dense(level, x, 1)
    c = level.coords
    y = b.expand(level.n, W.shape[2])
    for k, (dz, dy, dx) in enumerate(OFFS27):
        y = y + g[c[:, 0], c[:, 1] + 1 + dz, c[:, 2] + 1 + dy, c[:, 3] + 1 + dx] @ W[k]
    return y


def down2(fine: Level, coarse: Level, x, W, b):
    g = _dense(fine, x, 0)
    P = coarse.coords
    y = b.expand(coarse.n, W.shape[2])
    for j, (cz, cy, cx) in enumerate(CHILD8):
        y = y + g[P[:, 0], 2 * P[:, 1] + cz, 2 * P[:, 2] + cy, 2 * P[:, 3] + cx] @ W[j]
    return y


def up2(coarse: Level, fine: Level, z, W, b):
    zd = _dense(coarse, z, 0)                               # B, Dc, Hc, Wc, Cin
    B, Dc, Hc, Wc, _ = zd.shape
    cout = W.shape[2]
    parts = []
    for j, (cz, cy, cx) in enumerate(CHILD8):
        parts.append(zd @ W[j])                             # B, Dc, Hc, Wc, Cout
    t = torch.stack(parts, 0).reshape(2, 2, 2, B, Dc, Hc, Wc, cout)
    out = t.permute(3, 4, 0, 5, 1, 6, 2, 7).reshape(B, 2 * Dc, 2 * Hc, 2 * Wc, cout)
    c = fine.coords
    return b + out[c[:, 0], c[:, 1], c[:, 2], c[:, 3]]


def down3(fine: Level, coarse: Level, x, W, b):
    g = _dense(fine, x, 1)                                  # dense index = site + 1
    Q = coarse.coords
    y = b.expand(coarse.n, W.shape[2])
    for k, (kz, ky, kx) in enumerate(K27):                  # input 2q + k - 1 at dense index 2q + k
        y = y + g[Q[:, 0], 2 * Q[:, 1] + kz, 2 * Q[:, 2] + ky, 2 * Q[:, 3] + kx] @ W[k]
    return y


def up3(coarse: Level, fine: Level, z, W, b):
    zd = _dense(coarse, z, 0)                               # B, Dc, Hc, Wc, Cin
    B, Dc, Hc, Wc, _ = zd.shape
    out = torch.zeros((B, 2 * Dc + 1, 2 * Hc + 1, 2 * Wc + 1, W.shape[2]), dtype=zd.dtype)
    for k, (kz, ky, kx) in enumerate(K27):                  # output 2q + k - 1 at dense index 2q + k
        out[:, kz:kz + 2 * Dc:2, ky:ky + 2 * Hc:2, kx:kx + 2 * Wc:2] += zd @ W[k]
    c = fine.coords
    return b + out[c[:, 0], c[:, 1] + 1, c[:, 2] + 1, c[:, 3] + 1]


def head1(level: Level, x, W, b):
    return x @ W[0] + b


def build_levels(coords, dims, n_levels: int, strided3: bool = False) -> List[Level]:
    """Level 0 from the active coords, then each coarser level: the parents (2x2x2 stride-2 down
    convs) or, with strided3, the output set of a k = 3, stride 2, padding 1 convolution."""
    L = [Level(coords, dims)]
    for _ in range(n_levels - 1):
        L.append(L[-1].strided3() if strided3 else L[-1].parent())
    return L


def unet_is_k3(layers) -> bool:
    """Whether a U-Net's down / up convs are the k = 3 stride-2 pair."""
    return any(l.kind in ("down3", "up3") for l in layers)


def forward(layers, weights: Sequence[torch.Tensor], biases: Sequence[torch.Tensor],
            levels: List[Level], x: torch.Tensor, keep: Dict[str, torch.Tensor] = None):
    """Run a plain SubM3 stack or the sparse U-Net described by `layers` (npvs_inputs.Layer).
    `keep`, if given, receives every layer's output by layer name."""
    wi = {l.name: i for i, l in enumerate(layers)}

    def run(name, fn, *args):
        i = wi[name]
        l = layers[i]
        y = fn(*args, weights[i], biases[i])
        if l.relu:
            y = torch.relu(y)
        if keep is not None:
            keep[name] = y
        return y

    if "stem" not in wi:                      # plain stack
        a = x
        for l in layers:
            a = run(l.name, subm3, levels[0], a)
        return a
    nl = sum(1 for l in layers if l.kind in ("down2", "down3")) + 1
    k3 = unet_is_k3(layers)
    dn, upf = (down3, up3) if k3 else (down2, up2)
    a = run("stem", subm3, levels[0], x)
    skips = []
    for i in range(nl):
        a = run(f"enc{i}a", subm3, levels[i], a)
        a = run(f"enc{i}b", subm3, levels[i], a)
        skips.append(a)
        if i + 1 < nl:
            a = run(f"down{i}", lambda x_, W, b, i=i: dn(levels[i], levels[i + 1], x_, W, b), a)
    for i in range(nl - 2, -1, -1):
        a = run(f"up{i}", lambda x_, W, b, i=i: upf(levels[i + 1], levels[i], x_, W, b), a)
        a = a + skips[i]
        if keep is not None:
            keep[f"up{i}+skip"] = a
        a = run(f"dec{i}a", subm3, levels[i], a)
        a = run(f"dec{i}b", subm3, levels[i], a)
    return run("head", head1, levels[0], a)


def to_torch_params(ws, bs, requires_grad=False):
    W = [torch.tensor(np.asarray(w, dtype=np.float64), dtype=F64, requires_grad=requires_grad) for w in ws]
    B = [torch.tensor(np.asarray(b, dtype=np.float64), dtype=F64, requires_grad=requires_grad) for b in bs]
    return W, B
