"""Pins for the oracle's frustum setup, froxelization and ground truth (CPU only).

Each test checks the oracle against something other than itself: a closed form, a textbook
routine (slab ray/box intersection, searchsorted), an invariant the paper states (Sec. 3.2:
the displaced frustum encloses the viewcell's view; full occlusion; supp(V) within supp(G)),
or brute force.
"""
import dataclasses
import math

import numpy as np
import pytest

import npvs_inputs as I
from oracle import camera, froxel
from oracle.interleave import pack_bits, unpack_bits


def popcount(bits):
    return int(np.unpackbits(np.ascontiguousarray(bits).view(np.uint8)).sum())


# ------------------------------------------------------------------------------------------
# frustum (Sec. 3.2)
# ------------------------------------------------------------------------------------------

def test_frustum_basis_and_slices():
    vc = I.Viewcell(centre=(1.0, 2.0, 3.0), half=0.5, yaw=0.0)
    cam = camera.frustum(vc, 16)
    np.testing.assert_array_equal(cam.fwd, [0, 0, 1])
    np.testing.assert_array_equal(cam.right, [1, 0, 0])
    np.testing.assert_array_equal(cam.up, [0, 1, 0])
    assert cam.tan_half == np.float32(1.0)            # (60 + 2*15)/2 = 45 degrees
    delta = 0.5 / math.tan(math.radians(30)) + 0.5
    np.testing.assert_allclose(cam.origin, [1.0, 2.0, 3.0 - delta], rtol=0, atol=1e-6)
    z = cam.slices.astype(np.float64)
    assert z[0] == np.float32(0.1) and z[-1] == np.float32(100.0)
    ratio = z[1:] / z[:-1]
    np.testing.assert_allclose(ratio, (1000.0) ** (1 / 16), rtol=1e-6)
    # right-handed orthonormal basis for any yaw
    cam = camera.frustum(dataclasses.replace(vc, yaw=2.1), 16)
    r, u, f = (np.asarray(v, np.float64) for v in (cam.right, cam.up, cam.fwd))
    np.testing.assert_allclose(np.cross(r, u), f, atol=1e-7)
    np.testing.assert_allclose([r @ f, u @ f, r @ u], 0, atol=1e-7)


@pytest.mark.parametrize("yaw", [0.0, 0.7, 3.9])
def test_frustum_encloses_viewcell_views(yaw):
    """Sec. 3.2: every ray from a viewpoint in the viewcell, turned by up to beta beyond the
    FOV theta, stays inside the displaced frustum of half-angle (theta + 2 beta)/2."""
    vc = I.Viewcell(centre=(10.0, 2.0, -4.0), half=1.0, yaw=yaw)
    cam = camera.frustum(vc, 8)
    rng = np.random.default_rng(1)
    offs = rng.uniform(-1, 1, (4000, 3)) * vc.half
    offs[:8] = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]) * vc.half
    p = froxel.viewpoints(vc, cam, offs)
    tphi = float(cam.tan_half)
    ang = rng.uniform(-tphi, tphi, (len(p), 2))
    ang[:8] = tphi
    R = np.stack([cam.right, cam.up, cam.fwd]).astype(np.float64)
    d = np.concatenate([ang, np.ones((len(p), 1))], 1) @ R
    o = cam.origin.astype(np.float64)
    for t in (0.0, 0.3, 5.0, 80.0):
        v = (p + t * d - o) @ R.T
        assert (v[:, 2] > 0).all()
        assert (np.abs(v[:, 0]) <= v[:, 2] * tphi * (1 + 1e-6)).all()
        assert (np.abs(v[:, 1]) <= v[:, 2] * tphi * (1 + 1e-6)).all()


# ------------------------------------------------------------------------------------------
# froxelization (Sec. 3.2)
# ------------------------------------------------------------------------------------------

def point_camera(D=16, yaw=0.0, centre=(0.0, 0.0, 0.0)):
    vc = I.Viewcell(centre=centre, half=0.0, yaw=yaw)
    return camera.frustum(vc, D)


def test_slice_lookup_matches_searchsorted():
    cam = point_camera(D=24)
    z = cam.slices
    rng = np.random.default_rng(0)
    ts = np.concatenate([rng.uniform(0.0, 120.0, 500), z, np.nextafter(z, 0, dtype=np.float32)])
    for t in ts.astype(np.float32):
        ref = np.searchsorted(z, t, side="right") - 1
        ref = ref if (t >= z[0] and t < z[-1]) else -1
        assert froxel.slice_of(cam, float(t)) == ref


def test_fronto_parallel_quad_closed_form():
    """A quad at depth t0 facing the camera covers exactly the froxel columns whose pixel rays
    cross it, all in slice k(t0)."""
    W = H = 32
    D, s = 16, 4
    cam = point_camera(D)
    k0 = 9
    t0 = math.sqrt(float(cam.slices[k0]) * float(cam.slices[k0 + 1]))
    x_lo, x_hi, y_lo, y_hi = 5, 21, 11, 30
    ex = lambda i, n: t0 * (2.0 * i / n - 1.0)      # froxel boundary i at depth t0 (tan phi = 1)
    box = np.array([[ex(x_lo, W), ex(y_lo, H), t0, ex(x_hi, W), ex(y_hi, H), t0]], np.float32)
    for prec in (32, 64):
        bits = froxel.froxelize(cam, box, W, H, D, s, precision=prec)
        dense = unpack_bits(bits, W)
        exp = np.zeros((D, H, W), bool)
        exp[k0, y_lo:y_hi, x_lo:x_hi] = True
        np.testing.assert_array_equal(dense, exp)


def test_out_of_range_geometry_is_empty():
    W = H = 32
    D, s = 16, 2
    cam = point_camera(D)
    behind = [-5, -5, -10, 5, 5, -1]
    beyond = [-50, -50, 150, 50, 50, 160]
    outside = [200, -1, 5, 210, 1, 6]             # beyond the 45-degree side plane
    for b in (behind, beyond, outside):
        bits = froxel.froxelize(cam, np.array([b], np.float32), W, H, D, s)
        assert popcount(bits) == 0


def slab_reference(cam, boxes, W, H, D, s):
    """Textbook slab intersection (Kay-Kajiya) in float64: a ray through a box crosses its surface
    at t_enter = max_i min(t1_i, t2_i) and t_exit = min_i max(t1_i, t2_i); those are exactly the
    face hits, so each ray marks slice(t_enter) and slice(t_exit) when inside [z0, zD)."""
    sW, sH = s * W, s * H
    nx = (2 * np.arange(sW) + 1 - sW) / sW
    ny = (2 * np.arange(sH) + 1 - sH) / sH
    tp = float(cam.tan_half)
    f, r, u = (np.asarray(v, np.float64) for v in (cam.fwd, cam.right, cam.up))
    dirs = f + (nx[None, :, None] * tp) * r + (ny[:, None, None] * tp) * u
    o = cam.origin.astype(np.float64)
    z = cam.slices.astype(np.float64)
    dense = np.zeros((D, H, W), bool)
    for bx in boxes.astype(np.float64):
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (bx[:3] - o) / dirs
            t2 = (bx[3:] - o) / dirs
        tmin = np.minimum(t1, t2).max(-1)
        tmax = np.maximum(t1, t2).min(-1)
        hit = tmin <= tmax
        for t in (tmin, tmax):
            ok = hit & (t >= z[0]) & (t < z[-1])
            k = np.searchsorted(z, np.where(ok, t, z[0]), side="right") - 1
            bb, aa = np.nonzero(ok)
            dense[k[bb, aa], bb // s, aa // s] = True
    return pack_bits(dense)


@pytest.mark.parametrize("yaw", [0.0, 0.45, 2.6])
def test_froxelize_matches_slab_method(yaw):
    W = H = 32
    D, s = 24, 2
    vc = I.Viewcell(centre=(50.0, 8.0, 50.0), half=0.5, yaw=yaw)
    cam = camera.frustum(vc, D)
    boxes = I.random_boxes(seed=3, n=60)
    ref = slab_reference(cam, boxes, W, H, D, s)
    got64 = froxel.froxelize(cam, boxes, W, H, D, s, precision=64)
    got32 = froxel.froxelize(cam, boxes, W, H, D, s, precision=32)
    assert popcount(ref) > 100
    assert popcount(ref ^ got64) == 0
    # the binary32 mirror may differ only at ties on face edges / slice boundaries
    assert popcount(ref ^ got32) <= 1e-3 * popcount(ref) + 2


def test_columns_match_full_grid():
    boxes, vc = I.plain64_scene()
    cam = camera.frustum(vc, 32)
    full = unpack_bits(froxel.froxelize(cam, boxes, 64, 64, 32, 8), 64)   # D, H, W
    rng = np.random.default_rng(5)
    cols = np.stack([rng.integers(0, 64, 300), rng.integers(0, 64, 300)], 1)
    got = froxel.froxel_columns(cam, boxes, 64, 64, 32, 8, cols)
    for (x, y), w in zip(cols, got):
        ks = [k for k in range(32) if (w[k >> 5] >> (k & 31)) & 1]
        assert ks == list(np.nonzero(full[:, y, x])[0])


def test_plain64_scene_occupancy():
    boxes, vc = I.plain64_scene()
    cam = camera.frustum(vc, 32)
    G = froxel.froxelize(cam, boxes, 64, 64, 32, 8)
    occ = popcount(G) / (64 * 64 * 32)
    assert 0.03 < occ < 0.08


# ------------------------------------------------------------------------------------------
# ground truth (Sec. 3.2, last paragraph)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("precision", [64, 32])
def test_point_viewcell_is_zbuffer_visibility(precision):
    """h = 0, M = 1: the PVS is the froxel of each pixel ray's first hit (z-buffer), in binary64 and
    in the binary32 mirror."""
    W = H = 32
    D, s = 16, 2
    vc = I.Viewcell(centre=(50.0, 8.0, 20.0), half=0.0, yaw=0.3)
    cam = camera.frustum(vc, D)
    boxes = I.random_boxes(seed=7, n=50)
    raw, _ = froxel.gt_raycast(cam, boxes, W, H, D, s, froxel.viewpoints(vc, cam, np.zeros((1, 3))), precision)
    # z-buffer by slab intersection: nearest positive entry over boxes
    sW, sH = s * W, s * H
    nx = (2 * np.arange(sW) + 1 - sW) / sW
    ny = (2 * np.arange(sH) + 1 - sH) / sH
    f, r, u = (np.asarray(v, np.float64) for v in (cam.fwd, cam.right, cam.up))
    dirs = f + nx[None, :, None] * r + ny[:, None, None] * u
    o = cam.origin.astype(np.float64)
    best = np.full((sH, sW), np.inf)
    for bx in boxes.astype(np.float64):
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (bx[:3] - o) / dirs
            t2 = (bx[3:] - o) / dirs
        tmin = np.minimum(t1, t2).max(-1)
        tmax = np.maximum(t1, t2).min(-1)
        t = np.where(tmin > 0, tmin, tmax)
        ok = (tmin <= tmax) & (t > 0)
        best = np.where(ok & (t < best), t, best)
    z = cam.slices.astype(np.float64)
    dense = np.zeros((D, H, W), bool)
    ok = (best >= z[0]) & (best < z[-1])
    k = np.searchsorted(z, np.where(ok, best, z[0]), side="right") - 1
    bb, aa = np.nonzero(ok)
    dense[k[bb, aa], bb // s, aa // s] = True
    exp = pack_bits(dense)
    assert popcount(exp) > 100
    assert popcount(exp ^ raw) <= 2


@pytest.mark.parametrize("precision", [64, 32])
def test_full_occlusion(precision):
    """A wall spanning the whole frustum between the viewcell and a box hides the box."""
    W = H = 32
    D, s = 16, 2
    vc = I.Viewcell(centre=(0.0, 0.0, 0.0), half=0.5, yaw=0.0)
    cam = camera.frustum(vc, D)
    wall = [-500, -500, 6.0, 500, 500, 6.2]
    target = [-3, -3, 20.0, 3, 3, 25.0]
    boxes = np.array([wall, target], np.float32)
    G = froxel.froxelize(cam, boxes, W, H, D, s)
    G_target = froxel.froxelize(cam, np.array([target], np.float32), W, H, D, s)
    offs = I.gt_candidate_offsets(0, vc, 64)
    gt, raw = froxel.ground_truth(vc, cam, boxes, W, H, D, s, offs, 16, G, precision)
    assert popcount(G_target) > 0
    assert popcount(raw & G_target) == 0 and popcount(gt & G_target) == 0
    assert popcount(gt) > 0


@pytest.mark.parametrize("precision", [64, 32])
def test_monotone_in_viewpoints(precision):
    """Viewpoints of A a prefix of those of B (same frustum) => GT(A) within GT(B)."""
    W = H = 32
    D, s = 16, 2
    boxes, vc = I.plain64_scene()
    cam = camera.frustum(vc, D)
    G = froxel.froxelize(cam, boxes, W, H, D, 4)
    offs = I.gt_candidate_offsets(1, vc, 64)
    gA, _ = froxel.ground_truth(vc, cam, boxes, W, H, D, s, offs, 3, G, precision)
    gB, _ = froxel.ground_truth(vc, cam, boxes, W, H, D, s, offs, 12, G, precision)
    assert popcount(gA) > 0
    assert popcount(gA & ~gB) == 0
    assert popcount(gB & ~G) == 0


def test_gt_binary32_mirror_agrees_with_binary64_face_hits():
    """The binary32 mirror (slab entries, float32 viewpoints) against the binary64 nearest face hit
    on a city street viewcell: the same froxels up to ties at edges and slice bounds, and an empty
    scene or viewpoints facing away from every box give nothing."""
    W = H = 64
    D, s, M = 32, 1, 6
    boxes = I.city_boxes(1)
    vc = I.city_viewcells(1, 1, half=1.0)[0]
    cam = camera.frustum(vc, D)
    cand = froxel.viewpoints(vc, cam, I.gt_candidate_offsets(3, vc, 64))
    pts = cand[froxel.points_outside_boxes(cand, boxes)][:M]
    pts32 = pts.astype(np.float32).astype(np.float64)          # both sides from the same points
    r64, n64 = froxel.gt_raycast(cam, boxes, W, H, D, s, pts32, 64)
    r32, n32 = froxel.gt_raycast(cam, boxes, W, H, D, s, pts32, 32)
    n = popcount(r64)
    assert n > 500 and abs(n64 - n32) <= max(2, n64 // 1000)
    assert popcount(r64 ^ r32) <= max(3, n // 200), (popcount(r64 ^ r32), n)
    empty, nh = froxel.gt_raycast(cam, boxes[:0], W, H, D, s, pts32, 32)
    assert nh == 0 and popcount(empty) == 0
