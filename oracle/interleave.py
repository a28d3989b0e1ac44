"""Oracle 3-D volume-preserving interleave (test infrastructure; see ``oracle/__init__``).

Sec. 3.3, "3D volume-preserving interleaving": g_d splits the N_x x N_y x N_z grid into d x d x d
blocks and stacks the froxels of each block into one feature vector at the block's site of the
coarse grid (N_x/d x N_y/d x N_z/d); g_d^-1 inverts this.  V = g_d^-1(f_theta(g_d(G))).

Readings (the paper is silent on these):
  * Channel order inside a site: c * d^3 + (dz * d + dy) * d + dx, the 3-D analogue of
    pixel_unshuffle (the paper's codomain even omits the channel axis).
  * Input channels: c = 0 occupancy G in {0, 1}; c = 1 (when present) the normalised depth
    (k + 0.5) / D of slice k at occupied froxels and 0 elsewhere.
  * A coarse site is active (stored in the sparse tensor) iff any froxel of its block is
    occupied; active sites are listed in linear order of (b, z, y, x).
Grids are numpy arrays; bits use the layout [B][D][H][W/32], bit x & 31 of word x / 32.
"""
from __future__ import annotations

import numpy as np


def unpack_bits(bits: np.ndarray, W: int) -> np.ndarray:
    """[..., W/32] uint32 -> [..., W] bool (bit x & 31 of word x // 32)."""
    b = np.ascontiguousarray(bits, dtype="<u4").view(np.uint8)
    out = np.unpackbits(b, axis=-1, bitorder="little")
    return out[..., :W].astype(bool)


def pack_bits(dense: np.ndarray) -> np.ndarray:
    """[..., W] bool -> [..., W/32] uint32."""
    W = dense.shape[-1]
    assert W % 32 == 0
    by = np.packbits(dense.astype(np.uint8), axis=-1, bitorder="little")
    return np.ascontiguousarray(by).view("<u4").astype(np.uint32)


def g_d(dense: np.ndarray, d: int) -> np.ndarray:
    """Interleave a dense grid [B][D][H][W] (any dtype) -> [B][D/d][H/d][W/d][d^3]."""
    B, D, H, W = dense.shape
    assert D % d == 0 and H % d == 0 and W % d == 0
    t = dense.reshape(B, D // d, d, H // d, d, W // d, d)
    t = t.transpose(0, 1, 3, 5, 2, 4, 6)        # B, Z, Y, X, dz, dy, dx
    return t.reshape(B, D // d, H // d, W // d, d ** 3)


def g_d_inv(coarse: np.ndarray, d: int) -> np.ndarray:
    """De-interleave [B][Dc][Hc][Wc][d^3] -> [B][Dc*d][Hc*d][Wc*d]."""
    B, Dc, Hc, Wc, C = coarse.shape
    assert C == d ** 3
    t = coarse.reshape(B, Dc, Hc, Wc, d, d, d).transpose(0, 1, 4, 2, 5, 3, 6)
    return t.reshape(B, Dc * d, Hc * d, Wc * d)


def depth_channel(D: int) -> np.ndarray:
    """Normalised depth (k + 0.5) / D per slice, as the binary32 quotient (2k+1)/(2D)."""
    k = np.arange(D, dtype=np.float64)
    return ((2.0 * k + 1.0) / (2.0 * D)).astype(np.float32)


def interleave(G_bits: np.ndarray, W: int, d: int, in_ch: int):
    """Sparse interleave of a geometry grid.

    G_bits: [B][D][H][W/32].  Returns (coords [N][4] int32 (b, z, y, x) in linear order,
    feats [N][in_ch * d^3] float64, active [B][Dc][Hc][Wc] bool).
    """
    occ = unpack_bits(G_bits, W)                 # B, D, H, W
    B, D, H, _ = occ.shape
    chans = [g_d(occ.astype(np.float64), d)]
    if in_ch >= 2:
        dep = depth_channel(D).astype(np.float64)[None, :, None, None] * occ
        chans.append(g_d(dep, d))
    assert in_ch <= 2
    active = chans[0].any(axis=-1)
    idx = np.argwhere(active)                    # row-major = linear order (b, z, y, x)
    feats = np.concatenate([c[active] for c in chans], axis=-1)
    return idx.astype(np.int32), feats, active


def to_bf16_bits(x32: np.ndarray) -> np.ndarray:
    """binary32 -> bfloat16 bit patterns with round-to-nearest-even, in integer arithmetic.
    (Finite inputs only.)"""
    u = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)
    return r.astype(np.uint16)


def bf16_bits_to_f64(b: np.ndarray) -> np.ndarray:
    return (b.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def deinterleave(coords: np.ndarray, values: np.ndarray, B: int, D: int, H: int, W: int,
                 d: int) -> np.ndarray:
    """Scatter per-site vectors [N][d^3] back to a dense froxel grid [B][D][H][W]; inactive
    sites give 0."""
    coarse = np.zeros((B, D // d, H // d, W // d, d ** 3), dtype=values.dtype)
    c = coords.astype(np.int64)
    coarse[c[:, 0], c[:, 1], c[:, 2], c[:, 3]] = values
    return g_d_inv(coarse, d)


def pvs_from_logits(coords, logits, G_bits, W, d, tau: float = 0.5):
    """V = 1[sigmoid(f) >= tau] AND G (Sec. 3.1 threshold; Sec. 3.2 supp(V) within supp(G)),
    returned as bits [B][D][H][W/32] together with the dense probabilities."""
    B, D, H, _ = G_bits.shape
    p = 1.0 / (1.0 + np.exp(-np.asarray(logits, dtype=np.float64)))
    dense = deinterleave(coords, p, B, D, H, W, d)
    occ = unpack_bits(G_bits, W)
    return pack_bits((dense >= tau) & occ), dense
