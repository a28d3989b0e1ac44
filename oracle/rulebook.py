"""Oracle rulebooks (test infrastructure; see ``oracle/__init__``).

Sec. 2.3: a sparse tensor stores the active sites in a hash table; a submanifold convolution
visits, for every active site, the active sites at the 27 kernel offsets; a 2x2x2 stride-2
convolution maps every site p to its parent floor(p/2); a 3x3x3 stride-2 convolution with padding 1
dilates onto every q with p = 2q + k - 1. Written with a Python dict keyed by coordinates, straight
from those definitions.
"""
from __future__ import annotations

import numpy as np


def neighbour_map(coords: np.ndarray) -> np.ndarray:
    """nbr[n][k] = row of the site coords[n] + (dz, dy, dx), k = ((dz+1)*3 + (dy+1))*3 + (dx+1),
    or -1 if that site is not active."""
    pos = {tuple(c): i for i, c in enumerate(coords.tolist())}
    out = np.full((len(coords), 27), -1, dtype=np.int64)
    for n, (b, z, y, x) in enumerate(coords.tolist()):
        k = 0
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    out[n, k] = pos.get((b, z + dz, y + dy, x + dx), -1)
                    k += 1
    return out


def parent_level(coords: np.ndarray):
    """Parent sites {floor(p/2)} in linear order, the child rows of each parent (tap
    (cz*2+cy)*2+cx, -1 if absent) and, per child, parent_row * 8 + tap."""
    parents = sorted({(b, z // 2, y // 2, x // 2) for b, z, y, x in coords.tolist()})
    prow = {p: i for i, p in enumerate(parents)}
    down = np.full((len(parents), 8), -1, dtype=np.int64)
    up = np.zeros(len(coords), dtype=np.int64)
    for n, (b, z, y, x) in enumerate(coords.tolist()):
        p = prow[(b, z // 2, y // 2, x // 2)]
        tap = ((z % 2) * 2 + (y % 2)) * 2 + (x % 2)
        down[p, tap] = n
        up[n] = p * 8 + tap
    return np.asarray(parents, dtype=np.int64).reshape(-1, 4), down, up


def strided3_level(coords: np.ndarray, dims):
    """A stride-2 convolution with a 3^3 kernel and padding 1 (the k = 3, s = 2 downsampling of
    sparse backbones, Sec. 2.3): output site q of the halved grid receives input p = 2q + k - 1 through
    tap k = (kz*3 + ky)*3 + kx, k in {0,1,2}^3, so q is active iff one of those 27 inputs is (the
    dilated output set). Returns the output sites in linear order, down[q][k] = input row of
    2q + k - 1 (-1 if absent) and up[p][k] = output row q with p = 2q + k - 1 (-1 if no such q in the
    halved grid), the map of the transposed convolution."""
    B, Dz, Hy, Wx = dims
    half = (Dz // 2, Hy // 2, Wx // 2)
    pos = {tuple(c): i for i, c in enumerate(coords.tolist())}

    def sources(v, n):   # output coordinates q (and taps k) with v = 2q + k - 1 on one axis
        return [((v + 1 - k) // 2, k) for k in range(3) if (v + 1 - k) % 2 == 0 and 0 <= (v + 1 - k) // 2 < n]

    outs = set()
    for b, z, y, x in coords.tolist():
        for qz, _ in sources(z, half[0]):
            for qy, _ in sources(y, half[1]):
                for qx, _ in sources(x, half[2]):
                    outs.add((b, qz, qy, qx))
    outs = sorted(outs)
    orow = {q: i for i, q in enumerate(outs)}
    down = np.full((len(outs), 27), -1, dtype=np.int64)
    for i, (b, qz, qy, qx) in enumerate(outs):
        for kz in range(3):
            for ky in range(3):
                for kx in range(3):
                    down[i, (kz * 3 + ky) * 3 + kx] = pos.get((b, 2 * qz + kz - 1, 2 * qy + ky - 1, 2 * qx + kx - 1), -1)
    up = np.full((len(coords), 27), -1, dtype=np.int64)
    for n, (b, z, y, x) in enumerate(coords.tolist()):
        for qz, kz in sources(z, half[0]):
            for qy, ky in sources(y, half[1]):
                for qx, kx in sources(x, half[2]):
                    up[n, (kz * 3 + ky) * 3 + kx] = orow[(b, qz, qy, qx)]
    return np.asarray(outs, dtype=np.int64).reshape(-1, 4), down, up
