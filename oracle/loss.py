"""Oracle training loss, Adam and metrics in FP64 (test infrastructure; see ``oracle/__init__``).

Sec. 3.3 "Weighted Dice loss" and "Repulsive visibility loss"; Sec. 4.2 (lambda = 0.99,
learning rate 1e-3, "decay" 1e-10, tau = 0.5); Sec. 5.1 (FNR = FN / GTP, FPR = FP / GTP).

The paper's prose and formulas disagree: the prose calls a false negative a ground-truth froxel
missing from the prediction, while the printed sums attach the names the other way round, and the
printed attraction term 1 - FN/GTP would reward misses. Readings taken here, with y the ground
truth and p~ = p * g the soft prediction masked by the geometry grid g:
    TP = sum y p~,  FN = sum y (1 - p~) = GTP - TP,  FP = sum (1 - y) p~,  GTP = sum y
    L_dice = 1 - (2 TP + eps) / (2 TP + alpha FN + (1 - alpha) FP + eps)   (alpha weighs misses)
    L_attr = FN / (GTP + eps)   (= 1 - TP / (GTP + eps)),   L_rep = FP / (GTP + eps)
    L = lambda L_dice + (1 - lambda)(L_attr + L_rep) + w_bce * BCE,  averaged over the batch.
alpha (unspecified in the paper) = 0.9, eps = 1. BCE is not defined in the paper; where asked for
it is the mean binary cross-entropy with logits over occupied froxels, weight w_bce (default 0).
Sums run over the whole frame. Adam: beta1 0.9, beta2 0.999, eps 1e-8 (paper silent); the
paper's "decay 1e-10" is read as L2 weight decay added to the gradient.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from .interleave import g_d, unpack_bits


@dataclasses.dataclass(frozen=True)
class LossParams:
    alpha: float = 0.9
    eps: float = 1.0
    lam: float = 0.99
    w_bce: float = 0.0


def site_labels(bits: np.ndarray, coords: np.ndarray, W: int, d: int) -> np.ndarray:
    """Bits [B][D][H][W/32] -> {0,1} float64 [N][d^3] at the listed coarse sites, in the
    interleave channel order."""
    dense = unpack_bits(bits, W).astype(np.float64)
    c = g_d(dense, d)
    cc = coords.astype(np.int64)
    return c[cc[:, 0], cc[:, 1], cc[:, 2], cc[:, 3]]


def loss_terms(logits: torch.Tensor, coords: np.ndarray, G_bits: np.ndarray, GT_bits: np.ndarray,
               W: int, d: int, prm: LossParams = LossParams()):
    """Returns (L, terms) with terms[b] = dict(L, dice, attr, rep, bce, gtp, tp, fn, fp)."""
    B = G_bits.shape[0]
    y = torch.tensor(site_labels(GT_bits, coords, W, d), dtype=torch.float64)
    g = torch.tensor(site_labels(G_bits, coords, W, d), dtype=torch.float64)
    gtp_all = unpack_bits(GT_bits, W).reshape(B, -1).sum(1).astype(np.float64)
    p = torch.sigmoid(logits)
    pt = p * g
    bidx = torch.as_tensor(coords[:, 0].astype(np.int64))
    terms = []
    total = 0.0
    for b in range(B):
        sel = bidx == b
        yb, ptb, gb, zb = y[sel], pt[sel], g[sel], logits[sel]
        gtp = float(gtp_all[b])
        tp = (yb * ptb).sum()
        fn = gtp - tp
        fp = ((1.0 - yb) * ptb).sum()
        dice = 1.0 - (2.0 * tp + prm.eps) / (2.0 * tp + prm.alpha * fn + (1.0 - prm.alpha) * fp + prm.eps)
        attr = fn / (gtp + prm.eps)
        rep = fp / (gtp + prm.eps)
        nocc = gb.sum()
        if prm.w_bce != 0.0 and float(nocc) > 0:
            bce_el = torch.clamp(zb, min=0) - zb * yb + torch.log1p(torch.exp(-zb.abs()))
            bce = (bce_el * gb).sum() / nocc
        else:
            bce = torch.zeros((), dtype=torch.float64)
        Lb = prm.lam * dice + (1.0 - prm.lam) * (attr + rep) + prm.w_bce * bce
        total = total + Lb
        terms.append(dict(L=Lb, dice=dice, attr=attr, rep=rep, bce=bce, gtp=gtp, tp=tp, fn=fn, fp=fp))
    return total / B, terms


def adam_step(theta: np.ndarray, grad: np.ndarray, m: np.ndarray, v: np.ndarray, t: int,
              lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=1e-10):
    """One Adam step (t counts from 1). Returns (theta, m, v) in float64."""
    g = grad + wd * theta
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def rates(pvs_bits: np.ndarray, gt_bits: np.ndarray):
    """(FNR, FPR) = (FN / GTP, FP / GTP) over binary grids (Sec. 5.1)."""
    def pc(a):
        return int(np.unpackbits(np.ascontiguousarray(a).view(np.uint8)).sum())
    gtp = pc(gt_bits)
    fn = pc(gt_bits & ~pvs_bits)
    fp = pc(pvs_bits & ~gt_bits)
    return (fn / gtp if gtp else 0.0), (fp / gtp if gtp else 0.0)
