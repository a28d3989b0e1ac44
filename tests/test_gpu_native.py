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
                                                    ("nointerleave64", "bf16", 2, 0.2, True)])
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
