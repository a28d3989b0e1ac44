"""Train the 256x256x128 network on a pool of city viewcells and report missing geometry on held-out
cells (the paper's evaluation: FNR = missed ground-truth froxels / GTP, FPR = extra froxels / GTP,
Sec. 5.1), e.g.

    python -m paper_2509_24677_gb300.train_eval --steps 2000

Data (seeded, synthetic): 4 cities, 64 training and 16 held-out street viewcells of half-size 1 per
city; ground truth from 256 viewpoints per cell by GPU ray casting, ANDed with G. Batches of 8 cells
are drawn with a seeded sampler; every step is one replay of the captured training step (BF16
forward/backward, FP32 master weights, Adam). Prints one JSON line.

    --log steps.jsonl            one JSON line per --log-every steps (loss and its mean terms)
    --save ck.pt                 checkpoint at the end: trainer state, sampler state, step count
    --resume ck.pt --steps N     continue to N steps in all, with the checkpoint's parameters, Adam
                                 state, sampler state and kernel forms (same data flags); every step
                                 is deterministic, so this repeats the uninterrupted run's steps
                                 whenever that run used the same kernel forms
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

import npvs_inputs as I

from . import _lib as L
from . import data as Dm
from . import ops
from . import pipeline as P
from . import train as T


def _popcount(t: torch.Tensor) -> int:
    v = t.view(torch.uint8)
    table = torch.tensor([bin(i).count("1") for i in range(256)], dtype=torch.int64, device=t.device)
    return int(table[v.long()].sum().item())


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--train-per-scene", type=int, default=64)
    ap.add_argument("--eval-per-scene", type=int, default=16)
    ap.add_argument("--points", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--w-bce", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--log", default=None, help="append one JSON line per logged step to this file")
    ap.add_argument("--log-every", type=int, default=100)
    ap.add_argument("--save", default=None, help="write a checkpoint here after the last step")
    ap.add_argument("--resume", default=None, help="continue from a checkpoint written by --save")
    return ap.parse_args(argv)


def run(a, dev="cuda") -> dict:
    """Builds the data, trains, evaluates the held-out cells; returns the summary record."""
    wl = I.workload("city256")
    t0 = time.perf_counter()
    scenes = {s: I.city_boxes(s) for s in range(4)}
    cells = []  # (scene, viewcell, split)
    for s in range(4):
        vcs = I.city_viewcells(100 + s, a.train_per_scene + a.eval_per_scene, half=1.0)
        cells += [(s, v, "train") for v in vcs[:a.train_per_scene]]
        cells += [(s, v, "eval") for v in vcs[a.train_per_scene:]]
    # ground truth of every cell, 8 cells per GPU batch
    nb = len(scenes[0])
    words = wl.D * wl.H * (wl.W // 32)
    gts = torch.empty(len(cells), words, dtype=torch.int32, device=dev)
    cam_bytes = []
    for c0 in range(0, len(cells), 8):
        part = cells[c0:c0 + 8]
        b = Dm.make_batch([scenes[s] for s, _, _ in part], [v for _, v, _ in part], wl, a.points,
                          seed=a.seed + c0, device=dev)
        gts[c0:c0 + len(part)] = b.gt.view(len(part), words)
        cam_bytes.append(b.cams.view(len(part), -1))
    cams_all = torch.cat(cam_bytes)
    t_data = time.perf_counter() - t0

    ws, bs = I.kaiming_uniform(wl.layers, seed=a.seed)
    B = a.batch
    tr = T.Trainer(wl, wl.layers, ws, bs, B, L.BF16, loss_prm=ops.loss_params(w_bce=a.w_bce),
                   adam_prm=ops.adam_params(lr=a.lr), device=dev)
    boxes = torch.from_numpy(np.concatenate([scenes[0]] * B)).to(dev)
    offs = torch.arange(B + 1, dtype=torch.int32, device=dev) * nb
    cams = torch.empty(B * cams_all.shape[1], dtype=torch.uint8, device=dev)
    scene_dev = {s: torch.from_numpy(bx).to(dev) for s, bx in scenes.items()}
    train_idx = [i for i, c in enumerate(cells) if c[2] == "train"]
    eval_idx = [i for i, c in enumerate(cells) if c[2] == "eval"]
    rng = np.random.default_rng(a.seed)

    def load(ids):
        for e, i in enumerate(ids):
            boxes[e * nb:(e + 1) * nb].copy_(scene_dev[cells[i][0]])
        cams.view(B, -1).copy_(cams_all[ids])
        tr.gt.view(B, -1).copy_(gts[ids])

    done = 0                           # steps taken before this run
    if a.resume:
        ck = torch.load(a.resume, map_location="cpu", weights_only=False)
        tr.load_state_dict(ck["trainer"])  # parameters, Adam state and the tuned kernel forms
        rng.bit_generator.state = ck["rng"]
        done = int(ck["step"])
        if done >= a.steps:
            raise SystemExit(f"the checkpoint is at step {done}; ask for more --steps")
    load(list(rng.choice(train_idx, B, replace=False)))
    if not a.resume:
        tr.autotune(boxes, offs, cams)  # forward kernel forms for this batch size (no parameter update)
    g = tr.capture(boxes, offs, cams)  # its warm-up is step done + 1
    torch.cuda.synchronize()
    log_f = open(a.log, "a") if a.log else None

    def log_step(n):
        t = tr.terms.double().mean(0).tolist()
        log_f.write(json.dumps({"step": n, "loss": float(tr.loss.item()), "dice": t[L.LT_DICE],
                                "attr": t[L.LT_ATTR], "rep": t[L.LT_REP], "bce": t[L.LT_BCE]}) + "\n")

    if log_f and (done + 1) % a.log_every == 0:
        log_step(done + 1)
    losses = []
    t1 = time.perf_counter()
    for step in range(done + 1, a.steps):
        load(list(rng.choice(train_idx, B, replace=False)))
        g.replay()
        if step % 100 == 0 or step == a.steps - 1:
            losses.append((step + 1, round(float(tr.loss.item()), 5)))
        if log_f and ((step + 1) % a.log_every == 0 or step == a.steps - 1):
            log_step(step + 1)
    torch.cuda.synchronize()
    if log_f:
        log_f.close()
    if a.save:
        torch.save({"trainer": tr.state_dict(), "rng": rng.bit_generator.state, "step": a.steps, "args": vars(a)},
                   a.save)
    t_train = time.perf_counter() - t1
    if ops.npvs_check_status(tr.pipe.status) != 0:
        raise RuntimeError("device status set during training")

    # held-out evaluation through npvs_forward with the trained weights
    net = P.Net(wl.layers, [w.detach().cpu() for w in tr.params.w], [b.detach().cpu() for b in tr.params.b], dev)
    nf = P.NativeFrame(wl, net, 1, L.BF16, max_boxes=nb, device=dev)
    fn = fp = gtp = occ = 0
    for i in eval_idx:
        s, v, _ = cells[i]
        nf.run(scene_dev[s], torch.tensor([0, nb], dtype=torch.int32, device=dev), nb,
               cams_all[i].contiguous())
        gt = gts[i]
        fn += _popcount(gt & ~nf.pvs)
        fp += _popcount(nf.pvs & ~gt)
        gtp += _popcount(gt)
        occ += _popcount(nf.occ)
    out = {"steps": a.steps, "resumed_at": done, "batch": B, "train_cells": len(train_idx), "eval_cells": len(eval_idx),
           "gt_points": a.points, "lr": a.lr, "w_bce": a.w_bce, "data_seconds": round(t_data, 1),
           "train_seconds": round(t_train, 1), "steps_per_s": round((a.steps - 1 - done) / max(t_train, 1e-9), 1),
           "loss_curve": losses, "eval": {"FNR": round(fn / max(gtp, 1), 5), "FPR": round(fp / max(gtp, 1), 5),
                                          "GTP": gtp, "G_froxels": occ,
                                          "G_over_GT": round(occ / max(gtp, 1), 3)}}
    return out


def main(argv=None):
    print(json.dumps(run(parse_args(argv))), flush=True)


if __name__ == "__main__":
    main()
