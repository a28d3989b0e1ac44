"""GPU parity of npvs_prune (Sec. 3.2 occlusion culling by the PVS; Sec. 5.6 temporal bounding
volumes tested against the PVS) against the oracle: bit-exact keep / prune decisions.

Cases: the 64x64x32 plain scene against PVS sets of several densities (random subsets of G, G
itself, none, the PVS of a GPU frame), a ragged batch of three viewcells, empty and culled inputs,
and the full 256x256x128 (s = 8) city frame of the benchmark with its own PVS, sampled boxes
recomputed by the oracle and the whole box list checked against properties of the definition.
"""
import dataclasses

import numpy as np
import pytest
import torch

import npvs_inputs as I
from oracle import camera as ocam
from oracle import froxel as ofx
from oracle import interleave as oil

pytestmark = pytest.mark.gpu

DEV = "cuda"


def lib():
    from paper_2509_24677_gb300 import _lib, ops, pipeline
    return _lib, ops, pipeline


def gpu_prune(scenes, vcs, W, H, D, s, pvs):
    """pvs: uint32 [B][D][H][W/32]; returns uint8 [n_boxes] and the concatenated boxes."""
    L, ops, _ = lib()
    cams = [ops.npvs_camera_setup(v, D) for v in vcs]
    boxes = np.concatenate(scenes, 0).astype(np.float32) if len(scenes) else np.zeros((0, 6), np.float32)
    off = np.cumsum([0] + [len(b) for b in scenes]).astype(np.int32)
    vis = torch.full((max(len(boxes), 1),), 7, dtype=torch.uint8, device=DEV)
    ops.npvs_prune(torch.from_numpy(boxes).to(DEV), torch.from_numpy(off).to(DEV), ops.cameras_to_device(cams),
                   ops.grid(W, H, D, len(vcs)), s,
                   torch.from_numpy(np.ascontiguousarray(pvs).view(np.int32)).to(DEV), vis)
    torch.cuda.synchronize()
    return vis[:len(boxes)].cpu().numpy(), boxes


def test_prune_more_faces_than_the_fused_offsets():
    """The 12,000-building city (72,006 faces, more than the 65,536 whose offsets the item kernel adds
    itself) against a random 5 % subset of its G: the chunked scan path, box by box."""
    p = dataclasses.replace(I.CityParams(), n_buildings=12000, mu=2.3, sigma=0.7)
    boxes = I.city_boxes(2, p)
    vc = I.city_viewcells(2, 1, p, height=(2.0, 60.0))[0]
    W, H, D, s = 32, 32, 16, 2
    cam = ocam.frustum(vc, D)
    G = ofx.froxelize(cam, boxes, W, H, D, s)
    rng = np.random.default_rng(5)
    pvs = oil.pack_bits(oil.unpack_bits(G, W) & (rng.random((D, H, W)) < 0.05))
    ref = ofx.prune(cam, boxes, W, H, D, s, pvs)
    got, _ = gpu_prune([boxes], [vc], W, H, D, s, pvs[None])
    assert 6 * len(boxes) > 65536 and 0 < int(ref.sum()) < len(boxes)
    np.testing.assert_array_equal(got, ref)


def test_prune_plain64_bit_exact():
    boxes, vc = I.plain64_scene()
    W, H, D, s = 64, 64, 32, 8
    cam = ocam.frustum(vc, D)
    G = ofx.froxelize(cam, boxes, W, H, D, s)
    Gd = oil.unpack_bits(G, W)
    rng = np.random.default_rng(1)
    cases = {"none": np.zeros_like(Gd), "G": Gd}
    for frac in (0.002, 0.02, 0.2):
        cases[f"rand{frac}"] = Gd & (rng.random(Gd.shape) < frac)
    kept_counts = {}
    for name, dense in cases.items():
        pvs = oil.pack_bits(dense)
        ref = ofx.prune(cam, boxes, W, H, D, s, pvs)
        got, _ = gpu_prune([boxes], [vc], W, H, D, s, pvs[None])
        np.testing.assert_array_equal(got, ref, err_msg=name)
        kept_counts[name] = int(ref.sum())
    assert kept_counts["none"] == 0
    assert 0 < kept_counts["rand0.002"] < kept_counts["G"]


def test_prune_against_frame_pvs():
    """The PVS of a GPU frame of the plain network (random weights) as the test set."""
    L, ops, P = lib()
    wl = I.workload("plain64")
    boxes, vc = I.plain64_scene()
    ws, bs = I.kaiming_uniform(wl.layers, seed=0, bias_scale=0.05)
    net = P.Net(wl.layers, ws, bs, DEV)
    fp = P.FramePipeline(wl, net, 1, L.F32)
    cams = ops.cameras_to_device([ops.npvs_camera_setup(vc, wl.D)])
    bx = torch.from_numpy(boxes).to(DEV)
    off = torch.tensor([0, len(boxes)], dtype=torch.int32, device=DEV)
    fp.run(bx, off, cams)
    torch.cuda.synchronize()
    pvs = fp.pvs.cpu().numpy().view(np.uint32).reshape(wl.D, wl.H, wl.W // 32)
    ref = ofx.prune(ocam.frustum(vc, wl.D), boxes, wl.W, wl.H, wl.D, wl.supersample, pvs)
    got, _ = gpu_prune([boxes], [vc], wl.W, wl.H, wl.D, wl.supersample, pvs[None])
    np.testing.assert_array_equal(got, ref)


def test_prune_batched_ragged():
    p = dataclasses.replace(I.CityParams(), n_buildings=300)
    scenes = [I.city_boxes(0, p), I.city_boxes(1, p)[:170], I.city_boxes(2, p)[:5]]
    vcs = I.city_viewcells(0, 2, p) + I.city_viewcells(7, 1, p)
    W, H, D, s = 96, 40, 24, 3
    rng = np.random.default_rng(2)
    pvs = []
    for b in range(3):
        G = oil.unpack_bits(ofx.froxelize(ocam.frustum(vcs[b], D), scenes[b], W, H, D, s), W)
        pvs.append(oil.pack_bits(G & (rng.random(G.shape) < 0.05)))
    pvs = np.stack(pvs)
    got, _ = gpu_prune(scenes, vcs, W, H, D, s, pvs)
    start = 0
    for b in range(3):
        ref = ofx.prune(ocam.frustum(vcs[b], D), scenes[b], W, H, D, s, pvs[b])
        np.testing.assert_array_equal(got[start:start + len(scenes[b])], ref, err_msg=str(b))
        start += len(scenes[b])


def test_prune_empty_culled_and_unowned_boxes():
    L, ops, _ = lib()
    vc = I.Viewcell(centre=(0.0, 0.0, 0.0), half=0.5, yaw=0.0)
    W, H, D, s = 32, 32, 16, 2
    full = np.full((1, D, H, W // 32), 0xFFFFFFFF, np.uint32)
    behind = np.array([[-5, -5, -30, 5, 5, -10]], np.float32)
    got, _ = gpu_prune([behind], [vc], W, H, D, s, full)
    assert got.tolist() == [0]
    got, _ = gpu_prune([np.zeros((0, 6), np.float32)], [vc], W, H, D, s, full)
    assert got.size == 0
    # boxes before box_offsets[0] belong to no batch element: never kept
    cam = ops.npvs_camera_setup(vc, D)
    inview = np.array([[-1, -1, 5, 1, 1, 6], [-1, -1, 5, 1, 1, 6]], np.float32)
    vis = torch.full((2,), 9, dtype=torch.uint8, device=DEV)
    ops.npvs_prune(torch.from_numpy(inview).to(DEV), torch.tensor([1, 2], dtype=torch.int32, device=DEV),
                   ops.cameras_to_device([cam]), ops.grid(W, H, D, 1), s,
                   torch.from_numpy(full.view(np.int32)).to(DEV), vis)
    torch.cuda.synchronize()
    assert vis.cpu().tolist() == [0, 1]
    with pytest.raises(Exception):
        ops.npvs_prune(torch.from_numpy(inview).to(DEV), torch.tensor([0, 2], dtype=torch.int32, device=DEV),
                       ops.cameras_to_device([cam]), ops.grid(W, H, D, 1), 17,
                       torch.from_numpy(full.view(np.int32)).to(DEV), vis)


def test_prune_city256_full_size():
    """The 256x256x128 (s = 8) city frame of the benchmark with the PVS of its BF16 network (random
    weights: about half of G, so every box with a footprint is kept) and a sparse subset of it (1 %
    of its froxels, which prunes boxes): 40 sampled boxes recomputed by the oracle (kept and pruned
    ones), and for all 2,001 boxes: PVS subsets keep subsets, G keeps exactly the boxes with a
    footprint (the boxes an all-ones PVS keeps)."""
    L, ops, P = lib()
    wl = I.workload("city256")
    boxes, vc = I.city_boxes(0), I.city_viewcells(0, 1)[0]
    ws, bs = I.kaiming_uniform(wl.layers, seed=0, bias_scale=0.05)
    net = P.Net(wl.layers, ws, bs, DEV)
    fp = P.FramePipeline(wl, net, 1, L.BF16)
    cams = ops.cameras_to_device([ops.npvs_camera_setup(vc, wl.D)])
    bx = torch.from_numpy(boxes).to(DEV)
    off = torch.tensor([0, len(boxes)], dtype=torch.int32, device=DEV)
    fp.run(bx, off, cams)
    torch.cuda.synchronize()
    shape = (1, wl.D, wl.H, wl.W // 32)
    pvs = fp.pvs.cpu().numpy().view(np.uint32).reshape(shape)
    G = fp.occ.cpu().numpy().view(np.uint32).reshape(shape)
    rng = np.random.default_rng(0)
    sparse = oil.pack_bits(oil.unpack_bits(pvs[0], wl.W) & (rng.random((wl.D, wl.H, wl.W)) < 0.01))[None]
    args = ([boxes], [vc], wl.W, wl.H, wl.D, wl.supersample)
    v_pvs, _ = gpu_prune(*args, pvs)
    v_sp, _ = gpu_prune(*args, sparse)
    v_G, _ = gpu_prune(*args, G)
    v_all, _ = gpu_prune(*args, np.full(shape, 0xFFFFFFFF, np.uint32))
    assert np.all(v_sp <= v_pvs) and np.all(v_pvs <= v_G)
    np.testing.assert_array_equal(v_G, v_all)
    assert 0 < v_sp.sum() < v_G.sum() < len(boxes)
    kept, dropped = np.nonzero(v_sp)[0], np.nonzero(v_G & (1 - v_sp))[0]
    pick = np.concatenate([rng.choice(kept, min(20, len(kept)), replace=False),
                           rng.choice(dropped, min(20, len(dropped)), replace=False)])
    cam = ocam.frustum(vc, wl.D)
    for v, bits in ((v_sp, sparse[0]), (v_pvs, pvs[0])):
        ref = ofx.prune(cam, boxes[pick], wl.W, wl.H, wl.D, wl.supersample, bits)
        np.testing.assert_array_equal(v[pick], ref)
