"""Pins for the oracle's pruning (Sec. 3.2 occlusion culling by the PVS; Sec. 5.6 temporal bounding
volumes tested against the PVS), CPU only.

The oracle keeps a box iff its own froxels meet the PVS. It is checked against a closed form (a
fronto-parallel quad whose froxels are known in advance), against an independent froxelization
(the textbook slab method, which equals the binary64 oracle bit for bit), and against properties
of the definition: no PVS keeps nothing, geometry outside the frustum is never kept, keeping is
monotone in the PVS and distributes over a union of PVS sets.
"""
import math

import numpy as np
import pytest

import npvs_inputs as I
from oracle import camera, froxel
from oracle.interleave import pack_bits, unpack_bits
from test_oracle_froxel import point_camera, slab_reference


def pvs_from_dense(dense):
    return pack_bits(dense)


def test_prune_fronto_parallel_quad_closed_form():
    """The quad at depth t0 covers froxel columns [x_lo, x_hi) x [y_lo, y_hi) of slice k0 only:
    one PVS froxel inside that set keeps it; one just outside it (next column, next row, next
    slice) does not."""
    W = H = 32
    D, s = 16, 4
    cam = point_camera(D)
    k0 = 9
    t0 = math.sqrt(float(cam.slices[k0]) * float(cam.slices[k0 + 1]))
    x_lo, x_hi, y_lo, y_hi = 5, 21, 11, 30
    ex = lambda i, n: t0 * (2.0 * i / n - 1.0)
    box = np.array([[ex(x_lo, W), ex(y_lo, H), t0, ex(x_hi, W), ex(y_hi, H), t0]], np.float32)
    cases = [((k0, y_lo, x_lo), 1), ((k0, y_hi - 1, x_hi - 1), 1), ((k0, 20, 12), 1),
             ((k0, y_lo, x_hi), 0), ((k0, y_lo - 1, x_lo), 0), ((k0 + 1, 20, 12), 0), ((k0 - 1, 20, 12), 0)]
    for prec in (32, 64):
        for (k, y, x), want in cases:
            dense = np.zeros((D, H, W), bool)
            dense[k, y, x] = True
            got = froxel.prune(cam, box, W, H, D, s, pvs_from_dense(dense), precision=prec)
            assert got.tolist() == [want], ((k, y, x), prec)


def test_prune_empty_pvs_and_out_of_range_boxes():
    W = H = 32
    D, s = 16, 2
    cam = point_camera(D)
    boxes = np.array([[-5, -5, -10, 5, 5, -1],       # behind the camera
                      [-50, -50, 150, 50, 50, 160],  # beyond the far plane
                      [200, -1, 5, 210, 1, 6],       # outside the 45-degree side plane
                      [-1, -1, 5, 1, 1, 6]], np.float32)  # in view
    none = np.zeros((D, H, W // 32), np.uint32)
    full = np.full((D, H, W // 32), 0xFFFFFFFF, np.uint32)
    assert froxel.prune(cam, boxes, W, H, D, s, none).tolist() == [0, 0, 0, 0]
    assert froxel.prune(cam, boxes, W, H, D, s, full).tolist() == [0, 0, 0, 1]


@pytest.mark.parametrize("yaw", [0.0, 1.1])
def test_prune_matches_slab_method_binary64(yaw):
    """Per box, the slab-method froxels ANDed with a random PVS decide the same as the oracle in
    binary64 (where the two froxelizations are equal)."""
    W = H = 32
    D, s = 24, 2
    vc = I.Viewcell(centre=(50.0, 8.0, 50.0), half=0.5, yaw=yaw)
    cam = camera.frustum(vc, D)
    boxes = I.random_boxes(seed=11, n=40)
    rng = np.random.default_rng(4)
    geo = unpack_bits(slab_reference(cam, boxes, W, H, D, s), W)
    for frac in (0.02, 0.2):
        pvs_dense = geo & (rng.random(geo.shape) < frac)
        pvs = pvs_from_dense(pvs_dense)
        ref = np.array([1 if np.any(unpack_bits(slab_reference(cam, boxes[i:i + 1], W, H, D, s), W) & pvs_dense)
                        else 0 for i in range(len(boxes))], np.uint8)
        got = froxel.prune(cam, boxes, W, H, D, s, pvs, precision=64)
        np.testing.assert_array_equal(got, ref)
        assert 0 < ref.sum() < len(boxes)    # the case separates kept and pruned boxes


def test_prune_monotone_and_distributes_over_union():
    boxes, vc = I.plain64_scene()
    W, H, D, s = 64, 64, 32, 4
    cam = camera.frustum(vc, D)
    G = unpack_bits(froxel.froxelize(cam, boxes, W, H, D, s), W)
    rng = np.random.default_rng(8)
    A = G & (rng.random(G.shape) < 0.01)
    B = G & (rng.random(G.shape) < 0.01)
    va = froxel.prune(cam, boxes, W, H, D, s, pvs_from_dense(A))
    vb = froxel.prune(cam, boxes, W, H, D, s, pvs_from_dense(B))
    vab = froxel.prune(cam, boxes, W, H, D, s, pvs_from_dense(A | B))
    vA_sub = froxel.prune(cam, boxes, W, H, D, s, pvs_from_dense(A & (rng.random(G.shape) < 0.5)))
    np.testing.assert_array_equal(vab, va | vb)
    assert np.all(vA_sub <= va)
    # PVS = G keeps exactly the boxes with a footprint
    vg = froxel.prune(cam, boxes, W, H, D, s, pvs_from_dense(G))
    foot = np.array([popc(froxel.froxelize(cam, boxes[i:i + 1], W, H, D, s)) > 0 for i in range(len(boxes))])
    np.testing.assert_array_equal(vg.astype(bool), foot)
    assert 0 < va.sum() < vg.sum()


def popc(bits):
    return int(np.unpackbits(np.ascontiguousarray(bits).view(np.uint8)).sum())
