"""Oracle rulebooks (test infrastructure; see ``oracle/__init__``).

Sec. 2.3: a sparse tensor stores the active sites in a hash table; a submanifold convolution
visits, for every active site, the active sites at the 27 kernel offsets; a stride-2 convolution
maps every site p to its parent floor(p/2). Written with a Python dict keyed by coordinates,
straight from those definitions.
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
