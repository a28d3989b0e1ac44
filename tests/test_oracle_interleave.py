"""Pins for the oracle's interleave g_d, its inverse and the bit layout (CPU only; Sec. 3.3)."""
import itertools

import numpy as np
import pytest
import torch

from oracle import interleave as IL


def test_bit_layout():
    dense = np.zeros((1, 2, 3, 64), bool)
    dense[0, 1, 2, 33] = True
    bits = IL.pack_bits(dense)
    assert bits.shape == (1, 2, 3, 2)
    assert bits[0, 1, 2, 1] == 2 and bits.sum() == 2
    np.testing.assert_array_equal(IL.unpack_bits(bits, 64), dense)


@pytest.mark.parametrize("d", [1, 2, 4, 8, 32])
def test_roundtrip_and_bijection(d):
    rng = np.random.default_rng(d)
    B, D, H, W = 2, 2 * d, 3 * d, 2 * d
    x = rng.normal(size=(B, D, H, W))
    np.testing.assert_array_equal(IL.g_d_inv(IL.g_d(x, d), d), x)
    idx = np.arange(x.size).reshape(x.shape)
    perm = IL.g_d(idx, d).ravel()
    assert np.array_equal(np.sort(perm), np.arange(x.size))      # a permutation


def test_channel_order_by_loops():
    """Feature c*d^3 + (dz*d + dy)*d + dx of site (Z, Y, X) is froxel (d X + dx, d Y + dy, d Z + dz)."""
    d = 2
    rng = np.random.default_rng(0)
    dense = rng.random((1, 4, 4, 32)) < 0.2
    dense[0, 0, 0, :2] = True
    bits = IL.pack_bits(dense)
    coords, feats, active = IL.interleave(bits, 32, d, 2)
    Dn = 4
    n = 0
    for Z, Y, X in itertools.product(range(2), range(2), range(16)):
        blk = dense[0, d * Z:d * Z + d, d * Y:d * Y + d, d * X:d * X + d]
        if not blk.any():
            continue
        assert tuple(coords[n]) == (0, Z, Y, X)
        for dz, dy, dx in itertools.product(range(d), repeat=3):
            ch = (dz * d + dy) * d + dx
            occ = dense[0, d * Z + dz, d * Y + dy, d * X + dx]
            assert feats[n, ch] == float(occ)
            dep = (d * Z + dz + 0.5) / Dn if occ else 0.0
            assert feats[n, d ** 3 + ch] == pytest.approx(dep, abs=0, rel=1e-7)
        n += 1
    assert n == len(coords)


def test_d1_is_the_list_of_occupied_froxels():
    """Without interleave (d = 1, Sec. 5.4's ablation) the active sites are the occupied froxels in
    linear order, each with occupancy 1 and its slice-centre depth (k + 1/2) / D."""
    rng = np.random.default_rng(3)
    B, D, H, W = 2, 5, 3, 64
    dense = rng.random((B, D, H, W)) < 0.1
    coords, feats, active = IL.interleave(IL.pack_bits(dense), W, 1, 2)
    occ = [(b, z, y, x) for b in range(B) for z in range(D) for y in range(H) for x in range(W) if dense[b, z, y, x]]
    assert [tuple(c) for c in coords] == occ
    assert feats.shape == (len(occ), 2)
    assert (feats[:, 0] == 1.0).all()
    for (b, z, y, x), dep in zip(occ, feats[:, 1]):
        assert dep == np.float32((z + 0.5) / D)


def test_depth_channel_exact():
    for D in (32, 128, 192):
        v = IL.depth_channel(D)
        np.testing.assert_array_equal(v.astype(np.float64),
                                      np.array([(k + 0.5) / D for k in range(D)], np.float32))


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=20000), rng.uniform(0, 1, 20000),
                        IL.depth_channel(192)]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(IL.to_bf16_bits(x), ref)


def test_pvs_threshold_and_mask():
    d, W = 2, 32
    rng = np.random.default_rng(3)
    dense = rng.random((1, 4, 4, W)) < 0.3
    bits = IL.pack_bits(dense)
    coords, feats, _ = IL.interleave(bits, W, d, 1)
    logits = rng.normal(size=(len(coords), d ** 3))
    pvs, prob = IL.pvs_from_logits(coords, logits, bits, W, d, 0.5)
    exp = np.zeros_like(dense)
    for n, (b, Z, Y, X) in enumerate(coords):
        for dz, dy, dx in itertools.product(range(d), repeat=3):
            z = logits[n, (dz * d + dy) * d + dx]
            exp[b, d * Z + dz, d * Y + dy, d * X + dx] = z >= 0.0
    np.testing.assert_array_equal(IL.unpack_bits(pvs, W), exp & dense)
