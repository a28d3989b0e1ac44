"""npvs_forward, the whole frame as one call, against the same frame built from the individual entry
points (FramePipeline): identical kernels in the same order, so identical bits."""
import numpy as np
import pytest
import torch

import npvs_inputs as I
from test_gpu_parity import DEV, lib

pytestmark = pytest.mark.gpu


def frames(name, dtype, batch, capacity_frac=1.0, tune=False):
    L, ops, P = lib()
    wl = I.workload(name)
    if name == "plain64":
        scenes_vcs = [I.plain64_scene()] * batch
    else:
        vcs = I.city_viewcells(0, batch)
        scenes_vcs = [(I.city_boxes(0), v) for v in vcs]
    ws, bs = I.kaiming_uniform(wl.layers, seed=0, bias_scale=0.05)
    net = P.Net(wl.layers, ws, bs, DEV)
    boxes = np.concatenate([s for s, _ in scenes_vcs]).astype(np.float32)
    off = torch.tensor(np.cumsum([0] + [len(s) for s, _ in scenes_vcs]), dtype=torch.int32, device=DEV)
    bx = torch.from_numpy(boxes).to(DEV)
    cams = ops.cameras_to_device([ops.npvs_camera_setup(v, wl.D) for _, v in scenes_vcs])
    fp = P.FramePipeline(wl, net, batch, dtype, capacity_frac=capacity_frac)
    if tune:
        fp.autotune(bx, off, cams, reps=2)
    fp.run(bx, off, cams)
    nf = P.NativeFrame(wl, net, batch, dtype, max_boxes=len(boxes), capacity_frac=capacity_frac,
                       tuned=fp.descs if tune else None)
    nf.run(bx, off, len(boxes), cams, want_probs=True)
    assert ops.npvs_check_status(fp.status) == 0 and ops.npvs_check_status(nf.status) == 0
    return wl, fp, nf


@pytest.mark.parametrize("name,dt,batch,frac,tune", [("plain64", "f32", 1, 1.0, False), ("plain64", "bf16", 2, 1.0, False),
                                                    ("city256", "bf16", 2, 0.5, True), ("city256", "f32", 1, 1.0, False),
                                                    ("nointerleave64", "bf16", 2, 0.2, True),
                                                    ("city256_k3", "bf16", 2, 1.0, True), ("city256_k3", "f32", 1, 1.0, False)])
def test_native_forward_equals_entry_point_sequence(name, dt, batch, frac, tune):
    L, ops, P = lib()
    wl, fp, nf = frames(name, L.F32 if dt == "f32" else L.BF16, batch, frac, tune)
    assert torch.equal(fp.occ, nf.occ)
    assert torch.equal(fp.pvs, nf.pvs)
    lv_of = fp._level_of_layers()
    for i, l in enumerate(wl.layers):
        rows, nr = nf.layer_output(i)
        n = int(nr.item())
        assert n == int(fp.levels[lv_of[l.name]].n_rows.item())
        assert torch.equal(rows[:n], fp.acts[l.name][:n]), l.name
    n0 = int(fp.levels[0].n_rows.item())
    probs_ref = torch.sigmoid(fp.logits[:n0].double()).float()
    assert torch.allclose(nf.probs[:n0], probs_ref, rtol=1e-6, atol=1e-7)


def test_native_forward_graph_replay():
    L, ops, P = lib()
    wl, fp, nf = frames("plain64", L.BF16, 1)
    pvs0 = nf.pvs.clone()
    nf.pvs.zero_()
    boxes, vc = I.plain64_scene()
    bx = torch.from_numpy(boxes).to(DEV)
    off = torch.tensor([0, len(boxes)], dtype=torch.int32, device=DEV)
    cams = ops.cameras_to_device([ops.npvs_camera_setup(vc, wl.D)])
    g = nf.capture(bx, off, len(boxes), cams)
    nf.pvs.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(nf.pvs, pvs0)


def test_native_forward_argument_errors():
    L, ops, P = lib()
    wl = I.workload("plain64")
    ws, bs = I.kaiming_uniform(wl.layers, seed=0)
    net = P.Net(wl.layers, ws, bs, DEV)
    nf = P.NativeFrame(wl, net, 1, L.F32, max_boxes=40)
    boxes, vc = I.plain64_scene()
    bx = torch.from_numpy(boxes).to(DEV)
    off = torch.tensor([0, len(boxes)], dtype=torch.int32, device=DEV)
    cams = ops.cameras_to_device([ops.npvs_camera_setup(vc, wl.D)])
    with pytest.raises(L.NpvsError) as e:
        ops.npvs_forward(nf.desc, bx, off, len(boxes), cams, nf.occ, nf.pvs, None, nf.status, nf.ws[:1024])
    assert e.value.status == L.ERR_WORKSPACE
    with pytest.raises(L.NpvsError) as e:
        ops.npvs_forward(nf.desc, bx, off, 41, cams, nf.occ, nf.pvs, None, nf.status, nf.ws)
    assert e.value.status == L.ERR_INVALID_ARG


# ------------------------------------------------------------------------------------------
# the layer chain: the coarse levels' layers in one persistent launch (npvs_net_desc.chain_level)
# ------------------------------------------------------------------------------------------

def chained_frames(name, batch, chain_level, tune=False, capacity_frac=1.0):
    """The same frame through the entry points (the chained layers in the product form, which the
    chain computes) and through npvs_forward with chain_level."""
    L, ops, P = lib()
    wl = I.workload(name)
    vcs = I.city_viewcells(0, batch)
    boxes = np.concatenate([I.city_boxes(0)] * batch).astype(np.float32)
    nb = len(boxes) // batch
    off = torch.tensor([nb * i for i in range(batch + 1)], dtype=torch.int32, device=DEV)
    bx = torch.from_numpy(boxes).to(DEV)
    cams = ops.cameras_to_device([ops.npvs_camera_setup(v, wl.D) for v in vcs])
    ws, bs = I.kaiming_uniform(wl.layers, seed=0, bias_scale=0.05)
    net = P.Net(wl.layers, ws, bs, DEV)
    fp = P.FramePipeline(wl, net, batch, L.BF16, capacity_frac=capacity_frac)
    if tune:
        fp.autotune(bx, off, cams, reps=2)
    fp.use_chain_forms(chain_level)
    fp.run(bx, off, cams)
    nf = P.NativeFrame(wl, net, batch, L.BF16, max_boxes=len(boxes), tuned=fp.descs, chain_level=chain_level,
                       capacity_frac=capacity_frac)
    nf.run(bx, off, len(boxes), cams)
    assert ops.npvs_check_status(fp.status) == 0 and ops.npvs_check_status(nf.status) == 0
    return wl, fp, nf, (bx, off, cams, len(boxes))


@pytest.mark.parametrize("batch,chain_level,tune", [(1, 1, True), (1, 2, False), (1, 3, False), (2, 1, False)])
def test_chain_equals_product_form_layers(batch, chain_level, tune):
    """Every layer's output and the PVS of the chained frame are bitwise those of the layers launched
    one by one (the chained ones in the product form): same MMAs, same fixed-order reductions."""
    L, ops, P = lib()
    wl, fp, nf, _ = chained_frames("city256", batch, chain_level, tune)
    chained = P.chain_layer_indices(wl.layers, chain_level)
    assert len(chained) == {1: 16, 2: 10, 3: 4}[chain_level]
    lv_of = fp._level_of_layers()
    for i, l in enumerate(wl.layers):
        rows, nr = nf.layer_output(i)
        n = int(nr.item())
        assert n == int(fp.levels[lv_of[l.name]].n_rows.item()) and n > 0
        assert torch.equal(rows[:n], fp.acts[l.name][:n]), l.name
    assert torch.equal(fp.pvs, nf.pvs)


def test_chain_graph_replay_and_repeat_calls():
    """The chained frame captured in a CUDA graph and replayed, and called again eagerly, gives the
    same bits each time (the grid-barrier words go back to zero after every launch)."""
    L, ops, P = lib()
    wl, fp, nf, (bx, off, cams, n) = chained_frames("city256", 1, 1)
    pvs0 = nf.pvs.clone()
    out0 = nf.layer_output(len(wl.layers) - 2)[0].clone()
    g = nf.capture(bx, off, n, cams)
    for _ in range(3):
        nf.pvs.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(nf.pvs, pvs0)
    nf.run(bx, off, n, cams)
    assert ops.npvs_check_status(nf.status) == 0
    assert torch.equal(nf.pvs, pvs0) and torch.equal(nf.layer_output(len(wl.layers) - 2)[0], out0)


def test_chain_wait_timeout_is_reported_and_recoverable():
    """Under a one-cycle wait bound the chained frame returns with NPVS_ERR_TIMEOUT (its CTAs stop,
    pay the arrivals they owe to the grid barriers, drain and free their tensor memory); with the
    default bound and a zero-filled workspace the same frame is bitwise correct again. The frame's
    other convolutions run in the product form, whose copies are all issued and drained by one
    thread."""
    L, ops, P = lib()
    wl, fp, nf, (bx, off, cams, n) = chained_frames("city256", 1, 1)
    pvs0 = nf.pvs.clone()
    prev = ops.npvs_set_wait_limit(1)
    try:
        nf.pvs.zero_()
        nf.run(bx, off, n, cams)
        st = ops.npvs_check_status(nf.status)
    finally:
        ops.npvs_set_wait_limit(0)
    assert prev == 4_000_000_000 and st == L.ERR_TIMEOUT
    nf.ws.zero_()
    nf.run(bx, off, n, cams)
    assert ops.npvs_check_status(nf.status) == 0
    assert torch.equal(nf.pvs, pvs0)


def test_chain_level_argument_errors():
    """A chain level without a level below it, or over layers off the tensor-core shapes, is refused."""
    L, ops, P = lib()
    wl = I.workload("city256")
    ws, bs = I.kaiming_uniform(wl.layers, seed=0)
    net = P.Net(wl.layers, ws, bs, DEV)
    with pytest.raises((L.NpvsError, ValueError)):
        P.NativeFrame(wl, net, 1, L.BF16, max_boxes=10, chain_level=4)
    with pytest.raises((L.NpvsError, ValueError)):
        P.NativeFrame(wl, net, 1, L.F32, max_boxes=10, chain_level=1)


@pytest.mark.parametrize("chain_level,dtype", [(0, "bf16"), (1, "bf16"), (0, "f32")])
def test_empty_frame_and_a_frame_behind_the_camera(chain_level, dtype):
    """Frames with no active site: no boxes at all, and one box behind the camera, in a batch with a
    normal viewcell. Every launch of the frame (the layer chain included) runs on zero rows for the
    empty elements; their occupancy and PVS are all zero, the normal element equals the same frame
    run alone, and no status is raised."""
    L, ops, P = lib()
    wl = I.workload("city256")
    dt = L.BF16 if dtype == "bf16" else L.F32
    ws, bs = I.kaiming_uniform(wl.layers, seed=0, bias_scale=0.05)
    net = P.Net(wl.layers, ws, bs, DEV)
    vc_city = I.city_viewcells(0, 1)[0]
    city = I.city_boxes(0)
    behind = np.array([[-5, -5, -30, 5, 5, -10]], np.float32)
    vc0 = I.Viewcell(centre=(0.0, 0.0, 0.0), half=0.5, yaw=0.0)
    words = wl.D * wl.H * (wl.W // 32)

    def run(scenes, vcs):
        boxes = np.concatenate(scenes).astype(np.float32) if sum(len(s) for s in scenes) else np.zeros((1, 6), np.float32)
        bx = torch.from_numpy(boxes).to(DEV)
        off = torch.tensor(np.cumsum([0] + [len(s) for s in scenes]), dtype=torch.int32, device=DEV)
        cams = ops.cameras_to_device([ops.npvs_camera_setup(v, wl.D) for v in vcs])
        nf = P.NativeFrame(wl, net, len(vcs), dt, max_boxes=max(1, len(boxes)), chain_level=chain_level)
        nf.run(bx, off, int(off[-1].item()), cams)
        assert ops.npvs_check_status(nf.status) == 0
        return nf

    empty = np.zeros((0, 6), np.float32)
    nf = run([empty], [vc0])
    assert int(nf.occ.count_nonzero().item()) == 0 and int(nf.pvs.count_nonzero().item()) == 0
    nf = run([behind, city, empty], [vc0, vc_city, vc0])
    occ, pvs = nf.occ.view(3, words), nf.pvs.view(3, words)
    for b in (0, 2):
        assert int(occ[b].count_nonzero().item()) == 0 and int(pvs[b].count_nonzero().item()) == 0
    alone = run([city], [vc_city])
    assert torch.equal(occ[1], alone.occ.view(words))
    assert int(pvs[1].count_nonzero().item()) > 0
    # the batch's layers see the same rows for the one non-empty element, so its PVS is the same
    assert torch.equal(pvs[1], alone.pvs.view(words))
