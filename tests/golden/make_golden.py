"""Writes the oracle regression fixtures in this folder (run: python tests/golden/make_golden.py).

The paper prints no worked example of its per-frame computation (only timings and error rates), so
these fixtures are not paper values: they are outputs of the oracle itself on the seeded 64x64x32
scene, written by this script, which calls only the oracle and the seeded input generators. They
guard the oracle against unintended changes; the oracle's correctness is pinned separately by the
closed forms, textbook routines and invariants of tests/test_oracle_*.py.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import npvs_inputs as I  # noqa: E402
from oracle import camera as ocam  # noqa: E402
from oracle import froxel as ofx  # noqa: E402
from oracle import interleave as oil  # noqa: E402
from oracle import loss as olo  # noqa: E402
from oracle import network as onet  # noqa: E402


def compute() -> dict:
    wl = I.workload("plain64")
    boxes, vc = I.plain64_scene()
    cam = ocam.frustum(vc, wl.D)
    G = ofx.froxelize(cam, boxes, wl.W, wl.H, wl.D, wl.supersample)[None]
    dense = oil.unpack_bits(G[0], wl.W)
    coords, feats, _ = oil.interleave(G, wl.W, wl.d, wl.in_ch)
    ws, bs = I.kaiming_uniform(wl.layers, seed=0, bias_scale=0.05)
    levels = onet.build_levels(coords, (1, wl.D // wl.d, wl.H // wl.d, wl.W // wl.d), 1)
    W_, B_ = onet.to_torch_params(ws, bs)
    with torch.no_grad():
        logits = onet.forward(list(wl.layers), W_, B_, levels, torch.tensor(feats))
    pvs, _ = oil.pvs_from_logits(coords, logits.numpy(), G, wl.W, wl.d)
    # a ground truth for the loss: the G froxels of the even depth slices
    gt = G.copy()
    gt[:, 1::2] = 0
    L, terms = olo.loss_terms(logits, coords, G, gt, wl.W, wl.d, olo.LossParams(w_bce=1.0))
    t0 = terms[0]
    return {
        "about": "oracle outputs on the seeded plain64 scene (regression fixtures, not paper values)",
        "occupied_per_slice": [int(v) for v in dense.reshape(wl.D, -1).sum(1)],
        "occupied": int(dense.sum()),
        "active_sites": int(len(coords)),
        "coords_checksum": int((coords.astype(np.int64) * np.array([1, 7919, 104729, 1299709])).sum()),
        "logits_sum": float(logits.sum()),
        "logits_abs_sum": float(logits.abs().sum()),
        "logits_first": [float(v) for v in logits.reshape(-1)[:8]],
        "pvs_froxels": int(oil.unpack_bits(pvs[0], wl.W).sum()),
        "loss": {k: float(t0[k]) for k in ("L", "dice", "attr", "rep", "bce", "gtp", "tp", "fn", "fp")},
        "loss_total": float(L),
    }


if __name__ == "__main__":
    out = os.path.join(HERE, "oracle_plain64.json")
    with open(out, "w") as f:
        json.dump(compute(), f, indent=1)
    print("wrote", out)
