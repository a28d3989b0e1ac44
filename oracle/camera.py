"""Oracle viewcell -> frustum setup (test infrastructure; see ``oracle/__init__``).

Sec. 3.2, first paragraph: the frustum of a viewpoint c' displaced backwards by r / tan(theta/2)
encloses the PVS of lateral motion up to r; rotations up to beta on either side widen the field
of view to theta + 2 beta. Sec. 3.1: the frustum is split into a froxel grid.

Readings (the paper is silent on these):
  * Cube viewcell of half-size h: lateral radius r = h, and the apex is moved back by a further
    h so the whole cube (including its depth extent) lies in front of the apex:
    c' = c - f (h / tan(theta/2) + h).
  * Yaw about +y only, pitch 0: f = (sin psi, 0, cos psi), r = (cos psi, 0, -sin psi), u = (0,1,0).
  * Square viewport (Sec. 4.2 uses a 1:1 aspect ratio): half-angle phi = (theta + 2 beta)/2 in
    both x and y.
  * Depth slices spaced exponentially: z_k = near * (far/near)^(k/D), k = 0..D. (The supplement
    mentions linear and logarithmic depth scaling; the workloads here fix exponential.)
All arithmetic is binary64; the results are rounded once to binary32.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Camera:
    origin: np.ndarray   # c' (float32 [3])
    right: np.ndarray
    up: np.ndarray
    fwd: np.ndarray
    tan_half: np.float32  # tan(phi)
    slices: np.ndarray   # float32 [D+1]


def frustum(vc, D: int) -> Camera:
    theta = math.radians(vc.fov_deg)
    beta = math.radians(vc.rot_deg)
    phi = 0.5 * (theta + 2.0 * beta)
    psi = vc.yaw
    f = np.array([math.sin(psi), 0.0, math.cos(psi)])
    r = np.array([math.cos(psi), 0.0, -math.sin(psi)])
    u = np.array([0.0, 1.0, 0.0])
    delta = vc.half / math.tan(0.5 * theta) + vc.half
    c = np.asarray(vc.centre, dtype=np.float64)
    origin = c - delta * f
    z = [vc.near * math.pow(vc.far / vc.near, k / D) for k in range(D + 1)]
    f32 = lambda a: np.asarray(a, dtype=np.float64).astype(np.float32)
    return Camera(f32(origin), f32(r), f32(u), f32(f), np.float32(math.tan(phi)), f32(z))
