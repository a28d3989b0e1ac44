"""Training batches on the device: viewcells of seeded procedural scenes with their geometry grids
and ray-cast ground truth (Sec. 3.2 targets, Sec. 4.1 data generation).

The ground truth of a viewcell is the from-region PVS estimated by npvs_gt_raycast from M
viewpoints sampled uniformly in the cell (points inside a box are rejected and the first M
accepted are kept, so a smaller sample is a prefix of a larger one), ANDed with the cell's
geometry grid G. Viewpoint selection runs on the host; froxelization and ray casting run on the
GPU.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np
import torch

import npvs_inputs as I

from . import _lib as L
from . import ops


def viewpoints(vc, cam: L.Camera, boxes: np.ndarray, M: int, seed: int, oversample: int = 4) -> np.ndarray:
    """First M of the seeded candidate points of the cube cell that lie in no (closed) box,
    as world positions float32 [M][3]. The cell is aligned with the camera basis."""
    n = max(M * oversample, M + 64)
    off = I.gt_candidate_offsets(seed, vc, n)
    basis = np.array([list(cam.right), list(cam.up), list(cam.fwd)], dtype=np.float64)
    pts = np.asarray(vc.centre, dtype=np.float64)[None, :] + off @ basis
    lo = boxes[:, :3].astype(np.float64)
    hi = boxes[:, 3:].astype(np.float64)
    inside = np.zeros(len(pts), dtype=bool)
    for i in range(0, len(pts), 256):
        p = pts[i:i + 256, None, :]
        inside[i:i + 256] = ((p >= lo[None]) & (p <= hi[None])).all(-1).any(-1)
    ok = pts[~inside]
    if len(ok) < M:
        raise ValueError(f"only {len(ok)} of {n} candidate viewpoints lie outside the geometry")
    return ok[:M].astype(np.float32)


@dataclasses.dataclass
class Batch:
    boxes: torch.Tensor        # float [n][6], the elements' boxes concatenated
    box_offsets: torch.Tensor  # int32 [B+1]
    cams: torch.Tensor         # npvs_camera [B] (bytes)
    gt: torch.Tensor           # uint32 bits [B][D][H][W/32] (as int32)
    n_points: int


def make_batch(scenes: Sequence[np.ndarray], vcs: Sequence, wl, M: int, s_gt: int = 1, seed: int = 0,
               device="cuda") -> Batch:
    """Batch element e is viewcell vcs[e] of scene scenes[e]."""
    B = len(vcs)
    cams = [ops.npvs_camera_setup(v, wl.D) for v in vcs]
    pts = np.stack([viewpoints(v, c, s, M, seed + e) for e, (v, c, s) in enumerate(zip(vcs, cams, scenes))])
    boxes = np.concatenate(scenes, 0).astype(np.float32)
    off = np.cumsum([0] + [len(s) for s in scenes]).astype(np.int32)
    g = L.Grid(wl.W, wl.H, wl.D, B)
    bx = torch.from_numpy(boxes).to(device)
    of = torch.from_numpy(off).to(device)
    cd = ops.cameras_to_device(cams, device)
    words = B * wl.D * wl.H * (wl.W // 32)
    occ = torch.empty(words, dtype=torch.int32, device=device)
    ops.npvs_froxelize(bx, of, cd, g, wl.supersample, occ)
    gt = torch.empty(words, dtype=torch.int32, device=device)
    ops.npvs_gt_raycast(bx, of, cd, torch.from_numpy(pts).to(device), g, s_gt, gt, g_bits=occ)
    return Batch(bx, of, cd, gt, M)


def city_training_set(n_scenes: int = 4, per_scene: int = 2, half: float = 1.0, seed: int = 0) -> List:
    """(scene boxes, viewcell) pairs: per_scene street viewcells of each of n_scenes seeded cities,
    cells of half-size `half` (2 x 2 x 2 world units for half = 1)."""
    out = []
    for s in range(n_scenes):
        boxes = I.city_boxes(seed + s)
        for v in I.city_viewcells(seed + s, per_scene, half=half):
            out.append((boxes, v))
    return out
