#!/usr/bin/env python
"""NeuralPVS hot-path benchmark: PVS frames/s and ms/frame at 256x256x128 froxels on one GB300.

A step is one frame of the whole per-frame path: frustum setup (host, precomputed per viewcell),
froxelization of a 2,001-box procedural city (s = 8), interleave (d = 4, occupancy + depth ->
128 channels), rulebooks of 4 levels, the sparse U-Net 32/64/128/256 (BF16 tensor cores, FP32
accumulation), de-interleave + sigmoid + threshold + G mask. Inputs (boxes, cameras) are resident
in HBM; L2 is flushed between timed steps. `e2e` repeats the measurement through the public API
with host buffers (box and camera upload, PVS bit download inside the timed region). The same
line reports the plain FP32 path, the roofline of the dominant kernel and the FP64 CPU oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica (the path has no exchange step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import npvs_inputs as I  # noqa: E402

METRIC = "PVS frames/s at 256x256x128 froxels (BF16 path)"
WORKLOAD = "city256"
N_VIEWCELLS = 8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-single-thread", action="store_true", help="skip the one-thread CPU-oracle estimate")
    ap.add_argument("--chain-level", type=int, default=-1,
                    help="layer chain level of the headline frame (-1: the fastest of 0..levels-1 on this GPU)")
    ap.add_argument("--frames-per-step", type=int, default=0,
                    help="frames timed per step (0: enough for about 1 s of timed frames over all steps)")
    ap.add_argument("--no-train", action="store_true", help="skip the training-step measurement")
    ap.add_argument("--no-quality", action="store_true",
                    help="skip the 2,000-step training run and its held-out missing-geometry rate")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-viewcell batched measurement")
    ap.add_argument("--no-highres", action="store_true", help="skip the 512x512x192 measurement")
    ap.add_argument("--no-paper256", action="store_true",
                    help="skip the 256^3 measurements (d=8, 16, 32, and d=1 without interleave)")
    ap.add_argument("--no-k3", action="store_true", help="skip the k = 3 stride-2 U-Net frame")
    ap.add_argument("--grid-only", default=None,
                    choices=["city512", "paper256", "paper256_d1", "paper256_d8", "paper256_d32", "city256_k3"],
                    help="measure only this grid workload and print its record (not the headline line)")
    ap.add_argument("--grid-batch", type=int, default=0, help="viewcells of the grid workload (0: its default)")
    ap.add_argument("--grid-capacity", type=float, default=0.0,
                    help="level capacity as a fraction of the sites (0: the workload's default)")
    ap.add_argument("--profile-frame", action="store_true",
                    help="after timing, run one eager frame of the tuned grid workload inside the NVTX range "
                         "npvs_profile_frame (for a profiler's NVTX filter)")
    ap.add_argument("--train-points", type=int, default=256, help="ground-truth viewpoints per viewcell")
    ap.add_argument("--save-tuned", default=None,
                    help="write the autotuned per-layer kernel configurations of the headline frame (of the "
                         "grid workload with --grid-only) (JSON)")
    ap.add_argument("--tuned", default=None,
                    help="use saved per-layer configurations instead of autotuning (a run under a profiler "
                         "would otherwise tune on the profiler's launch times); the headline frame defaults "
                         "to the configuration shipped in the package")
    ap.add_argument("--autotune", action="store_true",
                    help="autotune the headline frame's per-layer configuration instead of using the shipped one")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device) -> float:
    """The largest value of x over the ranks of the default process group (x itself without one):
    per-step times of the replicas, so that the whole-job rate uses the slowest rank."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def step_quantiles(times_ms) -> dict:
    """Median and 99th percentile (nearest rank) of per-frame times in milliseconds; with fewer than
    100 samples the 99th percentile is not defined by them and the maximum is given instead."""
    t = sorted(float(x) for x in times_ms)
    if not t:
        return {"p50": None, "n": 0}
    out = {"p50": round(statistics.median(t), 4), "n": len(t)}
    if len(t) >= 100:
        out["p99"] = round(t[min(len(t) - 1, max(0, -(-99 * len(t) // 100) - 1))], 4)
    else:
        out["max"] = round(t[-1], 4)
    return out


def frames_per_step(steps: int, est_ms: float, target_s: float = 1.0) -> int:
    """Frames timed per step so that the timed frames add up to about target_s (at least one)."""
    return max(1, int(np.ceil(target_s * 1e3 / max(steps, 1) / max(est_ms, 1e-3))))


def replica_rate(world: int, units_per_rank: float, ms_per_step: float) -> float:
    """Whole-job throughput of `world` replicas that each process `units_per_rank` units per step
    in `ms_per_step` milliseconds (the slowest rank's time)."""
    return world * units_per_rank * 1000.0 / ms_per_step


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9 and f[1].replace(".", "").isdigit():
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        reasons = set()
        for r in rows:
            for name, v in (("hw_slowdown", r[5]), ("hw_thermal_slowdown", r[6]), ("sw_thermal_slowdown", r[7]),
                            ("sw_power_cap", r[8])):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "reasons": sorted(reasons)}


# Measured DRAM traffic (reads + writes, all 34 launches) of one city256 frame (the frame of viewcell
# 5 of the bench's cycle: 10,375 active sites at level 0) with the layer chain at level 1 and the
# level-0 layers in the forms below (profiles/city256_bf16_frame_launches.md), and that frame's
# algorithmic bytes; tied to the kernels as they are, so it must be measured again (or removed)
# when they change.
FRAME_DRAM = {"chain_level": 1,
              "forms": {"stem": "product", "enc0a": "window3", "enc0b": "window3",
                        "dec0a": "window3-nosplit", "dec0b": "window3-nosplit", "head": "gather"},
              "dram_bytes": 70_190_336, "algorithmic_bytes": 53_287_380,
              # the convolution kernels alone (layer chain, 6 level-0 conv_tc launches, 1 gather-reduce)
              "conv_dram_bytes": 63_967_232, "conv_algorithmic_bytes": 40_092_672}
# the headline frame's per-layer configuration, autotuned on a GB300 (bench.py --save-tuned)
TUNED_HEADLINE = os.path.join(ROOT, "paper_2509_24677_gb300", "tuned", "city256_bf16.json")


def frame_traffic(tuned: dict, chain_level: int, convs_only: bool = False):
    """Measured DRAM bytes of one whole frame (or of its convolution kernels), and that frame's
    algorithmic bytes, when the frame runs in the configuration they were measured with; else
    (None, None)."""
    forms = {k: tuned_label(tuned[k][0]) for k in FRAME_DRAM["forms"] if k in tuned}
    if chain_level == FRAME_DRAM["chain_level"] and forms == FRAME_DRAM["forms"]:
        if convs_only:
            return FRAME_DRAM["conv_dram_bytes"], FRAME_DRAM["conv_algorithmic_bytes"]
        return FRAME_DRAM["dram_bytes"], FRAME_DRAM["algorithmic_bytes"]
    return None, None


def tuned_label(cfg: dict) -> str:
    """Short name of an autotuned BF16 layer configuration."""
    if cfg.get("tune_form") == 2:
        return "product-split" if cfg.get("tune_max_split", 0) > 1 else "product"
    name = {3: "window", 4: "window3", 2: "gather-cp.async"}.get(cfg.get("tune_gather", 0), "gather")
    if cfg.get("tune_max_split") == 1:
        name += "-nosplit"
    if cfg.get("tune_gather_warps") == 4:
        name += "-4w"
    if cfg.get("tune_stages", 0) > 0:   # a stage count set by hand
        name += f"-s{cfg['tune_stages']}"
    return name


def layer_algorithmic(fp, wl):
    """Per stage: (bytes, flops, bound) from the actual rulebooks of the last frame (algorithmic
    counts: each operand byte once, FLOPs = 2 * pairs * cin * cout)."""
    out = {}
    lv_of = fp._level_of_layers()
    n = [int(lv.n_rows.item()) for lv in fp.levels]
    b = 2 if fp.dtype == 1 else 4
    for l in wl.layers:
        li = lv_of[l.name]
        if l.kind == "subm3":
            nb = fp.levels[li].nbr[:n[li]]
            pairs = int((nb >= 0).sum().item())
            n_in = n_out = n[li]
            taps = 27
        elif l.kind == "down2":
            pairs = n[li - 1]
            n_in, n_out, taps = n[li - 1], n[li], 8
        elif l.kind == "up2":
            pairs = n[li]
            n_in, n_out, taps = n[li + 1], n[li], 8
        elif l.kind == "down3":        # pairs: the existing inputs of each coarse output's 27 taps
            pairs = int((fp.levels[li - 1].down[:n[li]] >= 0).sum().item())
            n_in, n_out, taps = n[li - 1], n[li], 27
        elif l.kind == "up3":          # the same pairs, seen from the fine rows
            pairs = int((fp.levels[li].up[:n[li]] >= 0).sum().item())
            n_in, n_out, taps = n[li + 1], n[li], 27
        else:
            pairs = n[li]
            n_in = n_out = n[li]
            taps = 1
        ob = 4 if l.kind == "head1" else b
        byts = n_in * l.cin * b + n_out * l.cout * ob + taps * l.cin * l.cout * b + 4 * taps * n_out
        if l.kind in ("up2", "up3"):   # the skip input
            byts += n_out * l.cout * b
        out["conv:" + l.name] = dict(bytes=byts, flops=2 * pairs * l.cin * l.cout)
    W, H, D = wl.W, wl.H, wl.D
    out["interleave"] = dict(bytes=W * H * D // 8 + n[0] * (wl.feat_ch * b + 16), flops=0)
    out["deinterleave"] = dict(bytes=n[0] * wl.d ** 3 * 4 + 2 * W * H * D // 8, flops=0)
    tot = sum(n)
    out["rulebooks"] = dict(bytes=16 * tot + 8 * tot + 27 * 8 * tot + 4 * 27 * tot, flops=0)
    return out


def make_frame_inputs(device):
    from paper_2509_24677_gb300 import ops
    wl = I.workload(WORKLOAD)
    boxes = I.city_boxes(0)
    vcs = I.city_viewcells(0, N_VIEWCELLS)
    cams = [ops.npvs_camera_setup(v, wl.D) for v in vcs]
    return wl, boxes, vcs, cams


def cpu_oracle_frame(vc_index: int = 0, G=None):
    """One whole frame of the FP64 / binary32-mirror oracle on the host cores, nothing sampled:
    froxelization of the full 256x256x128 grid at s = 8 (binary32 mirror, OpenMP over rows),
    interleave, the four levels and the U-Net (float64 torch), de-interleave + threshold + G mask
    (viewcell `vc_index` of the bench's cycle). With G given the froxelization is skipped (its time
    is then not in the result). Returns (ms per frame, ms per stage, G, logits, coords)."""
    from oracle import camera as ocam
    from oracle import froxel as ofx
    from oracle import interleave as oil
    from oracle import network as onet
    wl = I.workload(WORKLOAD)
    boxes = I.city_boxes(0)
    vc = I.city_viewcells(0, N_VIEWCELLS)[vc_index % N_VIEWCELLS]
    cam = ocam.frustum(vc, wl.D)
    ws, bs = I.kaiming_uniform(wl.layers, seed=0)
    W_, B_ = onet.to_torch_params(ws, bs)
    t0 = time.perf_counter()
    if G is None:
        G = ofx.froxelize(cam, boxes, wl.W, wl.H, wl.D, wl.supersample)[None]
    t1 = time.perf_counter()
    coords, feats, _ = oil.interleave(G, wl.W, wl.d, wl.in_ch)
    t2 = time.perf_counter()
    levels = onet.build_levels(coords, (1, wl.D // wl.d, wl.H // wl.d, wl.W // wl.d), 4)
    with torch.no_grad():
        logits = onet.forward(list(wl.layers), W_, B_, levels, torch.tensor(feats)).numpy()
    t3 = time.perf_counter()
    oil.pvs_from_logits(coords, logits, G, wl.W, wl.d)
    t4 = time.perf_counter()
    stages = {"froxelize": 1e3 * (t1 - t0), "interleave": 1e3 * (t2 - t1), "rulebooks+network": 1e3 * (t3 - t2),
              "deinterleave": 1e3 * (t4 - t3)}
    return 1e3 * (t4 - t0), {k: round(v, 1) for k, v in stages.items()}, G, logits, coords


def cpu_oracle_loss_ms(G, logits, coords) -> float:
    """The oracle's training loss on a frame's logits (G standing in for the ground truth), ms."""
    from oracle import loss as oloss
    wl = I.workload(WORKLOAD)
    t0 = time.perf_counter()
    with torch.no_grad():
        oloss.loss_terms(torch.from_numpy(logits), coords, G, G, wl.W, wl.d)
    return 1e3 * (time.perf_counter() - t0)


def cpu_oracle_single_thread_estimate(G_path: str, n_cols: int = 2048):
    """The oracle with one thread: froxelization of `n_cols` random froxel columns at s = 8 scaled
    to the grid's 65,536 columns, plus interleave, U-Net and de-interleave of the whole frame on the
    oracle's own G (read from G_path). Returns (ms per frame, ms per stage)."""
    from oracle import camera as ocam
    from oracle import froxel as ofx
    wl = I.workload(WORKLOAD)
    G = np.load(G_path)
    ms_rest, stages, _, _, _ = cpu_oracle_frame(0, G=G)
    cam = ocam.frustum(I.city_viewcells(0, N_VIEWCELLS)[0], wl.D)
    rng = np.random.default_rng(0)
    cols = np.stack([rng.integers(0, wl.W, n_cols), rng.integers(0, wl.H, n_cols)], 1)
    t0 = time.perf_counter()
    ofx.froxel_columns(cam, I.city_boxes(0), wl.W, wl.H, wl.D, wl.supersample, cols)
    t_frox = (time.perf_counter() - t0) * (wl.W * wl.H) / n_cols
    stages["froxelize"] = round(1e3 * t_frox, 1)
    return ms_rest + 1e3 * t_frox, stages


def cpu_oracle_single_thread(G):
    """cpu_oracle_single_thread_estimate in a child process with OMP_NUM_THREADS=1 and one torch
    thread. Returns (ms per frame, ms per stage), or None if the child fails."""
    fd, path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    np.save(path, G)
    code = ("import json, torch; torch.set_num_threads(1); import bench; "
            f"r = bench.cpu_oracle_single_thread_estimate({path!r}); print(json.dumps([r[0], r[1]]))")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=600)
        ms, stages = json.loads(out.stdout.strip().splitlines()[-1])
        return float(ms), stages
    except Exception:
        return None
    finally:
        os.unlink(path)


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def bench_config(world: int) -> dict:
    """The workload both arms measure (the same dict in the reference arm's line)."""
    return {"workload": "city256: 256x256x128 froxels (s=8), 2,001-box procedural city seed 0, "
                        f"{N_VIEWCELLS} street viewcells cycled, d=4 (128 ch), sparse U-Net 32/64/128/256",
            "batch": 1, "parallelism": "replicas" if world > 1 else "single"}


REFERENCE_BUDGET_S = 150.0


def run_reference(args):
    """The reference arm: the oracle (the paper has no code) running whole frames of the same
    workload on the host cores, nothing sampled or scaled: each step is one full frame. A full
    frame takes seconds, so the steps run are capped by a wall-clock budget and the line declares
    the steps and warm-up frames that actually ran."""
    ws_, rank, _ = dist_env()
    if rank != 0:
        return
    warm = min(args.warmup, 1)
    t0 = time.perf_counter()
    for i in range(warm):
        cpu_oracle_frame(i)
    times, stages_acc = [], {}
    per = None
    for i in range(args.steps):
        if per is not None and (time.perf_counter() - t0) + per > REFERENCE_BUDGET_S:
            break
        ms, stages, _, _, _ = cpu_oracle_frame(warm + i)
        times.append(ms)
        per = ms / 1e3
        for k, v in stages.items():
            stages_acc[k] = stages_acc.get(k, 0.0) + v
    n = len(times)
    ms = statistics.mean(times)
    fps = 1000.0 / ms
    cores = os.cpu_count()
    desc = (f"{n} whole frames of the FP64 / binary32-mirror oracle (froxelization of all 65,536 columns at "
            f"s=8, interleave, U-Net, de-interleave; nothing scaled), viewcells cycled as in the GPU arm")
    line = {"impl": "reference", "metric": METRIC, "value": round(fps, 5), "unit": "frames/s", "n_gpus": args.gpus,
            "steps": n, "warmup": warm, "steps_requested": args.steps, "warmup_requested": args.warmup,
            "ms_per_step": round(ms, 2), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": bench_config(1),
            "stage_ms": {k: round(v / n, 1) for k, v in stages_acc.items()},
            "cpu_baseline": {"value": round(fps, 5), "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": desc, "cpu_model": cpu_model()},
            "e2e": {"value": round(fps, 5), "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(time.perf_counter() - t0, 1)}
    print(json.dumps(line), flush=True)


def run_quality(dev):
    """The training run of paper_2509_24677_gb300.train_eval with its defaults (4 cities x 64 training
    and 16 held-out street viewcells of half-size 1, ground truth from 256 viewpoints per cell by GPU
    ray casting, 2,000 steps of batch 8, BF16, Adam lr 1e-3), then the held-out cells through
    npvs_forward: FNR = missed ground-truth froxels / ground-truth froxels (the paper's missing
    geometry), FPR = extra froxels / ground-truth froxels."""
    from paper_2509_24677_gb300 import train_eval
    t0 = time.perf_counter()
    out = train_eval.run(train_eval.parse_args([]), dev)
    out["seconds"] = round(time.perf_counter() - t0, 1)
    out["what"] = ("2,000 BF16 training steps on synthetic city viewcells (random-init weights), then FNR / FPR "
                   "of the thresholded PVS on 64 held-out cells against GPU ray-cast ground truth")
    out["ground_truth"] = ("npvs_gt_raycast (binary32), bit-exact against the oracle's binary32 mirror of the same "
                           "ray cast (tests/test_gpu_train.py); the mirror agrees with the oracle's binary64 ray cast "
                           "up to ties at face edges")
    return out


def run_train(args, dev, flush):
    """Training steps/s: the city256 network on batches of 8 viewcells (2x2x2 world units, two
    street cells of each of 4 seeded cities), weighted Dice + repulsive visibility loss + BCE,
    BF16 forward/backward on the tensor cores, FP32 master weights and Adam, one CUDA graph per
    step. Ground truth: GPU ray casting from `train_points` viewpoints per cell, ANDed with G."""
    from paper_2509_24677_gb300 import _lib as L
    from paper_2509_24677_gb300 import data as Dm
    from paper_2509_24677_gb300 import ops
    from paper_2509_24677_gb300 import train as T
    wl = I.workload(WORKLOAD)
    pairs = Dm.city_training_set(4, 2, half=1.0)
    t0 = time.perf_counter()
    batch = Dm.make_batch([p[0] for p in pairs], [p[1] for p in pairs], wl, M=args.train_points, device=dev)
    torch.cuda.synchronize()
    t_gt = time.perf_counter() - t0
    ws, bs = I.kaiming_uniform(wl.layers, seed=0)
    tr = T.Trainer(wl, wl.layers, ws, bs, len(pairs), L.BF16, loss_prm=ops.loss_params(w_bce=1.0), device=dev)
    tr.gt.copy_(batch.gt)
    tuned = tr.autotune(batch.boxes, batch.box_offsets, batch.cams)   # forward layers (untimed)
    l0 = ops.npvs_launch_count()
    g = tr.capture(batch.boxes, batch.box_offsets, batch.cams)
    launches = (ops.npvs_launch_count() - l0) // 2
    st = torch.cuda.current_stream()
    losses, ev = [], []
    for i in range(args.warmup + args.steps):
        s_ = torch.cuda.Event(enable_timing=True)
        e_ = torch.cuda.Event(enable_timing=True)
        s_.record(st)
        g.replay()
        e_.record(st)
        if i >= args.warmup:
            ev.append((s_, e_))
        if i == 0 or i == args.warmup + args.steps - 1:
            torch.cuda.synchronize()
            losses.append(float(tr.loss.item()))
    torch.cuda.synchronize()
    if ops.npvs_check_status(tr.pipe.status) != 0:
        raise RuntimeError("device status set during the training steps")
    ms = statistics.mean(s_.elapsed_time(e_) for s_, e_ in ev)
    n_act = int(tr.pipe.levels[0].n_rows.item())
    gt_bits = int(torch.bitwise_count(batch.gt).sum().item()) if hasattr(torch, "bitwise_count") else None
    return {"steps_per_s": round(1000.0 / ms, 3), "ms_per_step": round(ms, 3), "batch": len(pairs), "dtype": "bf16",
            "master": "fp32", "optimizer": "adam lr 1e-3", "loss": "dice(alpha 0.9)+rvl(lambda 0.99)+bce(w 1)",
            "loss_first_last": [round(losses[0], 5), round(losses[-1], 5)], "gpu_launches_per_step": int(launches),
            "active_sites_level0": n_act, "gt_points": args.train_points, "gt_seconds": round(t_gt, 2),
            "gt_bits": gt_bits, "graph": "one CUDA graph replay per step; working set > L2",
            "forward_autotuned": {k: tuned_label(v[0]) for k, v in tuned.items()}}


def batched_scenes():
    """Four seeded cities for the batched workload. The 2,000-building city tops out near 4 %
    occupancy, so the other three are denser (6,000 / 12,000 / 24,000 buildings, the denser two
    with the taller lognormal(2.3, 0.7) heights) to span the 1-15 % occupancy band."""
    import dataclasses
    specs = [(2000, 2.0, 0.6), (6000, 2.0, 0.6), (12000, 2.3, 0.7), (24000, 2.3, 0.7)]
    return {sc: I.city_boxes(sc, dataclasses.replace(I.CityParams(), n_buildings=nb, mu=mu, sigma=sg))
            for sc, (nb, mu, sg) in enumerate(specs)}


def select_batched_viewcells(dev, wl, scenes, n_pick=64, per_scene=512, lo=0.01, hi=0.15):
    """The batched-inference workload: a pool of street viewcells of the 4 cities with camera heights
    2-60 (to widen the occupancy range), froxelized on the GPU; the n_pick cells nearest to n_pick
    evenly spaced occupancy targets in [lo, hi] (each cell used once)."""
    from paper_2509_24677_gb300 import _lib as L
    from paper_2509_24677_gb300 import ops
    pool = []
    chunk = 64
    for sc, boxes in scenes.items():
        vcs = I.city_viewcells(sc, per_scene, height=(2.0, 60.0))
        rep = torch.from_numpy(np.concatenate([boxes] * chunk)).to(dev)
        off = torch.arange(chunk + 1, dtype=torch.int32, device=dev) * len(boxes)
        occ = torch.empty(chunk * wl.D * wl.H * (wl.W // 32), dtype=torch.int32, device=dev)
        for c0 in range(0, len(vcs), chunk):
            part = vcs[c0:c0 + chunk]
            cams = ops.cameras_to_device([ops.npvs_camera_setup(v, wl.D) for v in part]
                                         + [ops.npvs_camera_setup(part[-1], wl.D)] * (chunk - len(part)), dev)
            ops.npvs_froxelize(rep, off, cams, L.Grid(wl.W, wl.H, wl.D, chunk), wl.supersample, occ)
            bits = occ.view(chunk, -1).cpu().numpy().view(np.uint8)
            cnt = np.unpackbits(bits, axis=1).sum(1)
            for v, c in zip(part, cnt[:len(part)]):
                pool.append((sc, v, float(c) / (wl.W * wl.H * wl.D)))
    used, picked = set(), []
    for t in np.linspace(lo, hi, n_pick):
        best = min((i for i in range(len(pool)) if i not in used), key=lambda i: abs(pool[i][2] - t))
        used.add(best)
        picked.append(pool[best])
    return picked


def chain_levels_for(P, wl):
    """Chain levels the network allows: 0 (none) and every k whose chained layers are tensor-core
    shapes (cin % 32 == 0, cout % 16 == 0)."""
    if any(l.kind in ("down3", "up3") for l in wl.layers):
        return [0]                    # the layer chain runs the 2x2x2 pair only
    n_levels = 1 + sum(1 for l in wl.layers if l.kind == "down2")
    out = [0]
    for k in range(1, n_levels):
        idx = P.chain_layer_indices(wl.layers, k)
        if idx and all(wl.layers[i].cin % 32 == 0 and wl.layers[i].cout % 16 == 0 for i in idx):
            out.append(k)
    return out


def fastest_chain_frame(P, L, wl, net, B, descs, bx, of, nb, cams, dev, capacity_frac=1.0, reps=10):
    """The captured BF16 frame (npvs_forward) at each allowed chain level, timed over `reps` graph
    replays; returns (NativeFrame, graph, level, {level: median ms}) of the fastest."""
    st = torch.cuda.current_stream()
    best, times = None, {}
    for k in chain_levels_for(P, wl):
        nfk = P.NativeFrame(wl, net, B, L.BF16, max_boxes=nb, device=dev, tuned=descs, capacity_frac=capacity_frac,
                            chain_level=k)
        gk = nfk.capture(bx, of, nb, cams)
        ev = []
        for i in range(3 + reps):
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record(st)
            gk.replay()
            e_.record(st)
            if i >= 3:
                ev.append((s_, e_))
        torch.cuda.synchronize()
        times[k] = statistics.median(s_.elapsed_time(e_) for s_, e_ in ev)
        if best is None or times[k] < times[best[2]]:
            best = (nfk, gk, k)
        else:
            del gk, nfk
    return best[0], best[1], best[2], {str(k): round(v, 4) for k, v in times.items()}


def run_batched(args, dev, net, tuned):
    """64 viewcells of uneven occupancy in one batched frame (one launch per layer over the
    concatenated rulebooks, one CUDA graph of npvs_forward), and each viewcell alone as a
    single-frame graph replay for the per-viewcell latency distribution."""
    from paper_2509_24677_gb300 import _lib as L
    from paper_2509_24677_gb300 import ops, pipeline as P
    wl = I.workload(WORKLOAD)
    scenes = batched_scenes()
    picked = select_batched_viewcells(dev, wl, scenes)
    boxes = np.concatenate([scenes[sc] for sc, _, _ in picked]).astype(np.float32)
    off = np.cumsum([0] + [len(scenes[sc]) for sc, _, _ in picked]).astype(np.int32)
    bx = torch.from_numpy(boxes).to(dev)
    of = torch.from_numpy(off).to(dev)
    cams = ops.cameras_to_device([ops.npvs_camera_setup(v, wl.D) for _, v, _ in picked], dev)
    B = len(picked)
    frac = 0.6
    fpb = P.FramePipeline(wl, net, B, L.BF16, device=dev, capacity_frac=frac)
    tuned_b = fpb.autotune(bx, of, cams, reps=3)
    # stage split of the batch: a stage-timed graph of the same frame, entry point by entry point
    timer = P.StageTimer()
    gst = fpb.capture(bx, of, cams, timer=timer)
    acc = {}
    for i in range(4):
        gst.replay()
        torch.cuda.synchronize()
        if i >= 1:
            for k, v in timer.totals().items():
                acc[k] = acc.get(k, 0.0) + v / 3
    conv_ms = sum(v for k, v in acc.items() if k.startswith("conv:"))
    stages = {k: round(v, 3) for k, v in acc.items() if not k.startswith("conv:")}
    stages["convs (22 layers)"] = round(conv_ms, 3)
    del gst
    nfb, g, chain_b, chain_b_ms = fastest_chain_frame(P, L, wl, net, B, fpb.descs, bx, of, len(boxes), cams, dev,
                                                      capacity_frac=frac, reps=5)
    del fpb
    st = torch.cuda.current_stream()
    ts = []
    for i in range(3 + max(5, args.steps // 3)):
        s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_.record(st)
        g.replay()
        e_.record(st)
        if i >= 3:
            ts.append((s_, e_))
    torch.cuda.synchronize()
    if ops.npvs_check_status(nfb.status) != 0:
        raise RuntimeError("device status set in the batched frame")
    batch_ms = statistics.median(s_.elapsed_time(e_) for s_, e_ in ts)
    n_act = int(nfb.layer_output(-1)[1].item())
    del g, nfb
    # per-viewcell latency: each cell alone through one single-frame graph (buffers refilled per cell)
    nmax = max(len(v) for v in scenes.values())
    nf1 = P.NativeFrame(wl, net, 1, L.BF16, max_boxes=nmax, device=dev, tuned=tuned)
    bx1 = torch.zeros(nmax, 6, dtype=torch.float32, device=dev)
    of1 = torch.zeros(2, dtype=torch.int32, device=dev)
    cams_b = cams.view(B, -1)                 # one npvs_camera (bytes) per row
    cam1 = cams_b[0].clone()
    g1 = nf1.capture(bx1, of1, nmax, cam1)
    lat = []
    for k, (sc, v, _) in enumerate(picked):
        nbx = len(scenes[sc])
        bx1[:nbx].copy_(torch.from_numpy(scenes[sc]))
        of1[1] = nbx
        cam1.copy_(cams_b[k])
        rs = []
        for i in range(6):
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record(st)
            g1.replay()
            e_.record(st)
            if i >= 2:
                rs.append((s_, e_))
        torch.cuda.synchronize()
        lat.append(statistics.median(s_.elapsed_time(e_) for s_, e_ in rs))
    occs = [o for _, _, o in picked]
    return {"viewcells": B, "scenes": "4 cities of 2k/6k/12k/24k buildings, seeds 0-3",
            "stage_ms": dict(sorted(stages.items(), key=lambda kv: -kv[1])),
            "conv_layer_ms": {k[5:]: round(v, 3) for k, v in acc.items() if k.startswith("conv:")},
            "occupancy_range": [round(min(occs), 4), round(max(occs), 4)],
            "batch_ms": round(batch_ms, 4), "frames_per_s": round(B * 1000.0 / batch_ms, 2),
            "chain": {"level": chain_b, "ms_per_batch_by_level": chain_b_ms},
            "per_viewcell_ms": {"p50": round(float(np.percentile(lat, 50)), 4),
                                "p99": round(float(np.percentile(lat, 99)), 4), "max": round(max(lat), 4)},
            "active_sites_level0": n_act, "capacity_frac": frac,
            "autotuned": {k: tuned_label(v[0]) for k, v in tuned_b.items()}}


def run_highres(args, dev, tf_bf16, hbm_gbs):
    """512x512x192 froxels (s = 4), d = 8 (2 x 512 = 1024 input channels), U-Net 64/128/256/512,
    BF16, batch 4: four street viewcells of the 10,000-building city (heights lognormal(2.3, 0.7)).
    Per layer: achieved GB/s of the algorithmic bytes and TFLOP/s of the algorithmic FLOPs, from
    stage events captured in a graph of the same frame."""
    B = args.grid_batch or 4
    boxes = I.city_boxes(0, I.CITY_LARGE)
    vcs = I.city_viewcells(0, B, I.CITY_LARGE)
    return run_grid_workload(args, dev, tf_bf16, hbm_gbs, I.workload("city512"), boxes, vcs,
                             "city512: 512x512x192 froxels (s=4), d=8 (1024 ch), U-Net 64/128/256/512, "
                             f"10,000-building city seed 0, {B} viewcells")


def run_paper256(args, dev, tf_bf16, hbm_gbs):
    """The paper's grid and interleave factor: 256x256x256 froxels (s = 8), d = 16 (one occupancy
    channel, 4096 input channels per coarse site), stem submanifold conv 4096 -> 192 ("~200"),
    U-Net 192/256, head to 4096 logits; BF16, batch 1 (one viewcell of the 2,000-building city), as
    the paper's per-frame inference. Per layer: achieved GB/s and TFLOP/s of the algorithmic work."""
    boxes = I.city_boxes(0)
    vcs = I.city_viewcells(0, args.grid_batch or 1)
    return run_grid_workload(args, dev, tf_bf16, hbm_gbs, I.workload("paper256"), boxes, vcs,
                             "paper256: 256x256x256 froxels (s=8), d=16 (4096 ch), U-Net 192/256, "
                             "2,001-box city seed 0, 1 viewcell")


def run_paper256_d1(args, dev, tf_bf16, hbm_gbs):
    """The paper's "no interleave" ablation (Sec. 5.4, ablation table): the paper256 scene and U-Net
    (192/256) on the 256^3 froxel grid itself, d = 1, one occupancy channel per froxel (stem 1 ->
    192, head 256 -> 1 logit). Level capacities at 10 % of the sites (1.9 % are occupied)."""
    boxes = I.city_boxes(0)
    vcs = I.city_viewcells(0, args.grid_batch or 1)
    return run_grid_workload(args, dev, tf_bf16, hbm_gbs, I.workload("paper256_d1"), boxes, vcs,
                             "paper256_d1: 256x256x256 froxels (s=8), d=1 (1 ch), U-Net 192/256, "
                             "2,001-box city seed 0, 1 viewcell", capacity_frac=0.1)


def run_paper256_factor(args, dev, tf_bf16, hbm_gbs, d):
    """The paper's runtime-and-memory comparison over the interleaving factor (d in {8, 16, 32},
    Sec. 5 figure on runtime and peak memory): the paper256 scene and U-Net 192/256 at d = 8 (512
    input channels per coarse site, 32^3 coarse grid) or d = 32 (32,768 channels, 8^3 coarse grid;
    stem 32768 -> 192 and head 192 -> 32768)."""
    boxes = I.city_boxes(0)
    vcs = I.city_viewcells(0, args.grid_batch or 1)
    return run_grid_workload(args, dev, tf_bf16, hbm_gbs, I.workload(f"paper256_d{d}"), boxes, vcs,
                             f"paper256_d{d}: 256x256x256 froxels (s=8), d={d} ({d ** 3} ch), U-Net 192/256, "
                             "2,001-box city seed 0, 1 viewcell")


def run_city256_k3(args, dev, tf_bf16, hbm_gbs):
    """The headline scene and U-Net (256x256x128, d = 4, 32/64/128/256) with the backbone's k = 3,
    stride 2, padding 1 down convs (each coarser level the dilated output set) and their transposes
    in place of the 2x2x2 pair: one viewcell per frame, BF16, every layer its own launch."""
    boxes = I.city_boxes(0)
    vcs = I.city_viewcells(0, args.grid_batch or 1)
    return run_grid_workload(args, dev, tf_bf16, hbm_gbs, I.workload("city256_k3"), boxes, vcs,
                             "city256_k3: 256x256x128 froxels (s=8), d=4 (128 ch), U-Net 32/64/128/256 with k=3 "
                             "stride-2 down convs and their transposes, 2,001-box city seed 0")


def run_grid_workload(args, dev, tf_bf16, hbm_gbs, wl, boxes, vcs, label, capacity_frac=1.0):
    """Batch of len(vcs) viewcells of one scene through the BF16 frame (autotuned, one graph of
    npvs_forward), then stage and per-layer times from a stage-timed graph of the same frame.
    Also reports the peak device memory the frame objects held and the bytes of the layer outputs
    for the rows that are active."""
    from paper_2509_24677_gb300 import _lib as L
    from paper_2509_24677_gb300 import ops, pipeline as P
    if args.grid_capacity > 0:
        capacity_frac = args.grid_capacity
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    mem0 = torch.cuda.memory_allocated()
    B = len(vcs)
    bx = torch.from_numpy(np.concatenate([boxes] * B)).to(dev)
    of = torch.arange(B + 1, dtype=torch.int32, device=dev) * len(boxes)
    cams = ops.cameras_to_device([ops.npvs_camera_setup(v, wl.D) for v in vcs], dev)
    ws, bs = I.kaiming_uniform(wl.layers, seed=0)
    net = P.Net(wl.layers, ws, bs, dev)
    fp = P.FramePipeline(wl, net, B, L.BF16, device=dev, capacity_frac=capacity_frac)
    fp.run(bx, of, cams)
    stt = ops.npvs_check_status(fp.status)
    if stt != 0:
        raise RuntimeError(f"device status {stt:#x} set in the {wl.name} frame")
    if args.grid_only and args.tuned:            # the configuration a plain run saved (for profiling)
        with open(args.tuned) as fh:
            fp.apply_tuned(json.load(fh))
        tuned = {k: (v, float("nan")) for k, v in fp.tuned_configs().items()}
    else:
        tuned = fp.autotune(bx, of, cams, reps=3)
    if args.grid_only and args.save_tuned:
        with open(args.save_tuned, "w") as fh:
            json.dump(fp.tuned_configs(), fh)
    nf, g, chain_k, chain_ms = fastest_chain_frame(P, L, wl, net, B, fp.descs, bx, of, len(boxes) * B, cams, dev,
                                                   capacity_frac=capacity_frac, reps=5)
    st = torch.cuda.current_stream()
    ts = []
    for i in range(3 + max(5, args.steps // 3)):
        s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_.record(st)
        g.replay()
        e_.record(st)
        if i >= 3:
            ts.append((s_, e_))
    torch.cuda.synchronize()
    ms = statistics.median(s_.elapsed_time(e_) for s_, e_ in ts)
    del g, nf
    timer = P.StageTimer()
    gt = fp.capture(bx, of, cams, timer=timer)
    acc = {}
    for i in range(5):
        gt.replay()
        torch.cuda.synchronize()
        if i >= 2:
            for k, v in timer.totals().items():
                acc[k] = acc.get(k, 0.0) + v / 3
    alg = layer_algorithmic(fp, wl)
    per_layer = {}
    for k, v in alg.items():
        if k.startswith("conv:") and k in acc:
            t = acc[k] * 1e-3
            per_layer[k[5:]] = {"ms": round(acc[k], 4), "GB/s": round(v["bytes"] / t / 1e9, 1),
                                "TFLOP/s": round(v["flops"] / t / 1e12, 2),
                                "tensor_frac": round(v["flops"] / t / 1e12 / tf_bf16, 4)}
    profiled = None
    if args.profile_frame:
        # one eager frame of the tuned per-layer kernels, in layer order, bracketed for a profiler
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("npvs_profile_frame")
        fp.run(bx, of, cams)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        profiled = [[l.name, "simt" if l.cin % 8 or l.cout % 8 else tuned_label(tuned[l.name][0])]
                    for l in wl.layers]
    occ = float(np.unpackbits(fp.occ.cpu().numpy().view(np.uint8)).mean())
    n_lv = [int(lv.n_rows.item()) for lv in fp.levels]
    lv_of = fp._level_of_layers()
    act_bytes = sum(n_lv[lv_of[l.name]] * l.cout * (4 if l.kind == "head1" else 2) for l in wl.layers)
    peak_mb = (torch.cuda.max_memory_allocated() - mem0) / 2**20
    rec = {"workload": label, "batch": B, "ms_per_batch": round(ms, 3),
            "chain": {"level": chain_k, "ms_per_batch_by_level": chain_ms},
            "memory_mb": {"peak_device": round(peak_mb, 1), "layer_outputs_active": round(act_bytes / 2**20, 1)},
            "frames_per_s": round(B * 1000.0 / ms, 2), "occupancy": round(occ, 4),
            "active_sites": [int(lv.n_rows.item()) for lv in fp.levels],
            "stage_ms": {k: round(v, 4) for k, v in sorted(acc.items(), key=lambda kv: -kv[1]) if not k.startswith("conv:")},
            "conv_layers": per_layer, "peaks": {"hbm_gbs": hbm_gbs, "bf16_tflops": tf_bf16},
            "autotuned": {l.name: ("simt" if l.cin % 8 or l.cout % 8 else tuned_label(tuned[l.name][0]))
                          for l in wl.layers}, "capacity_frac": capacity_frac}
    if profiled:
        rec["profile_frame_layers"] = profiled
    return rec


def run_grid_only(args):
    """One grid workload on its own (its record as the printed line): for profiling one workload
    without the headline frame and the other measurements."""
    torch.cuda.set_device(0)
    dev = "cuda:0"
    hbm_gbs, tf_bf16, _ = load_peaks()
    name = args.grid_only
    if name == "city512":
        rec = run_highres(args, dev, tf_bf16, hbm_gbs)
    elif name == "paper256":
        rec = run_paper256(args, dev, tf_bf16, hbm_gbs)
    elif name == "paper256_d1":
        rec = run_paper256_d1(args, dev, tf_bf16, hbm_gbs)
    elif name == "city256_k3":
        rec = run_city256_k3(args, dev, tf_bf16, hbm_gbs)
    else:
        rec = run_paper256_factor(args, dev, tf_bf16, hbm_gbs, int(name.split("_d")[1]))
    print(json.dumps({"grid_only": name, **rec}), flush=True)


def run_ours(args):
    from paper_2509_24677_gb300 import _lib as L
    from paper_2509_24677_gb300 import ops, pipeline as P

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
        torch.cuda.set_device(local)
    else:
        torch.cuda.set_device(0)
    dev = f"cuda:{torch.cuda.current_device()}"
    wl, boxes, vcs, cams = make_frame_inputs(dev)
    ws, bs = I.kaiming_uniform(wl.layers, seed=0)
    net = P.Net(wl.layers, ws, bs, dev)
    boxes_d = torch.from_numpy(boxes).to(dev)
    off_d = torch.tensor([0, len(boxes)], dtype=torch.int32, device=dev)
    cams_d = [ops.cameras_to_device([c], dev) for c in cams]
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    hbm_gbs, tf_bf16, peak_src = load_peaks()

    fp = P.FramePipeline(wl, net, 1, L.BF16, device=dev)
    cam_buf = torch.empty_like(cams_d[0])
    cam_buf.copy_(cams_d[0])
    # untimed first frames (lazy weight packing, kernel attributes), then one CUDA graph per path
    fp.run(boxes_d, off_d, cam_buf)
    if ops.npvs_check_status(fp.status) != 0:
        raise RuntimeError("device status set on the first frame")
    if args.tuned is None and not args.autotune and os.path.exists(TUNED_HEADLINE):
        args.tuned = TUNED_HEADLINE
    if args.tuned:                                   # per-layer kernel configuration (untimed)
        with open(args.tuned) as fh:
            fp.apply_tuned(json.load(fh))
        tuned = {k: (v, float("nan")) for k, v in fp.tuned_configs().items()}
    else:
        tuned = fp.autotune(boxes_d, off_d, cam_buf)
    if args.save_tuned:
        with open(args.save_tuned, "w") as fh:
            json.dump(fp.tuned_configs(), fh)
    st = torch.cuda.current_stream()

    def timed_replays(graph, steps, warmup, per_step=None, mark_last=False, frames=1):
        """Per step `frames` frames, each after an L2 flush and timed alone with CUDA events on the
        launching stream; returns the per-frame times (ms) of the timed steps."""
        out = []
        for i in range(warmup + steps):
            for f in range(frames):
                flush.zero_()
                cam_buf.copy_(cams_d[(i * frames + f) % len(cams_d)])
                s = torch.cuda.Event(enable_timing=True)
                e = torch.cuda.Event(enable_timing=True)
                last = mark_last and i == warmup + steps - 1 and f == frames - 1
                if last:    # the last timed frame in an NVTX range "frame", for a profiler to select
                    torch.cuda.nvtx.range_push("frame")
                s.record(st)
                graph.replay()
                e.record(st)
                if last:
                    torch.cuda.nvtx.range_pop()
                if per_step is not None:
                    torch.cuda.synchronize()
                    if i >= warmup:
                        per_step()
                if i >= warmup:
                    out.append((s, e))
        torch.cuda.synchronize()
        return [s.elapsed_time(e) for s, e in out]

    # the timed frames go through the public single call npvs_forward (same kernels as fp). The
    # layer chain (the coarse levels' layers in one persistent launch, npvs_net_desc.chain_level)
    # is chosen by timing the captured frame at each level on this GPU (0: no chain)
    nb = len(boxes)
    chain_ms = {}
    levels = [args.chain_level] if args.chain_level >= 0 else list(range(0, fp.n_levels))
    for k in levels:
        nfk = P.NativeFrame(wl, net, 1, L.BF16, max_boxes=nb, device=dev, tuned=fp.descs, chain_level=k)
        gk = nfk.capture(boxes_d, off_d, nb, cam_buf)
        chain_ms[k] = statistics.median(timed_replays(gk, 30, 3))
        if ops.npvs_check_status(nfk.status) != 0:
            raise RuntimeError(f"device status set with chain level {k}")
        del gk, nfk
    chain_level = min(chain_ms, key=chain_ms.get)
    nf = P.NativeFrame(wl, net, 1, L.BF16, max_boxes=nb, device=dev, tuned=fp.descs, chain_level=chain_level)
    nf32 = P.NativeFrame(wl, net, 1, L.F32, max_boxes=nb, device=dev)
    l0 = ops.npvs_launch_count()
    g16 = nf.capture(boxes_d, off_d, nb, cam_buf)
    launches_per_frame = (ops.npvs_launch_count() - l0) // 2      # warm-up run + captured run
    g32 = nf32.capture(boxes_d, off_d, nb, cam_buf)
    timer = P.StageTimer()
    g16t = fp.capture(boxes_d, off_d, cam_buf, timer=timer)
    torch.cuda.synchronize()

    # ---- device-timed BF16 frames (the headline) ----------------------------------------------
    # a few untimed frames give the frame time that sizes the timed region (about 1 s of frames)
    est = statistics.median(timed_replays(g16, 5, 2))
    fps_step = frames_per_step(args.steps, est) if args.frames_per_step <= 0 else args.frames_per_step
    clocks = Clocks(torch.cuda.current_device())
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_bf16 = timed_replays(g16, args.steps, args.warmup, mark_last=True, frames=fps_step)
    clk = clocks.stop()
    launches_timed = launches_per_frame * args.steps * fps_step
    ms_frame = max_over_ranks(statistics.mean(t_bf16), dev)
    ms = ms_frame * fps_step
    if ops.npvs_check_status(nf.status) != 0:
        raise RuntimeError("device status set during the timed frames")

    # ---- per-stage times (stage events captured in a second graph of the same frame) ----------
    acc = {}

    def add_stage_times():
        for k, v in timer.totals().items():
            acc[k] = acc.get(k, 0.0) + v

    timed_replays(g16t, args.steps, 2, add_stage_times)
    stage_ms = {k: v / args.steps for k, v in acc.items()}

    # ---- FP32 path, same inputs ------------------------------------------------------------------
    t_f32 = timed_replays(g32, max(5, args.steps // 2), 2, frames=max(1, fps_step // 2))
    ms32 = statistics.mean(t_f32)

    # ---- end to end through the public API with host buffers -------------------------------------
    boxes_h = torch.from_numpy(boxes).pin_memory()
    cams_h = [ops.cameras_to_device([c], "cpu").pin_memory() for c in cams]
    pvs_h = torch.empty(nf.pvs.numel(), dtype=torch.int32).pin_memory()
    def e2e_frames(run_one, steps, warmup, frames):
        ev = []
        for i in range(warmup + steps):
            for f in range(frames):
                flush.zero_()
                s = torch.cuda.Event(enable_timing=True)
                e = torch.cuda.Event(enable_timing=True)
                s.record(st)
                boxes_d.copy_(boxes_h, non_blocking=True)
                run_one(cams_h[(i * frames + f) % len(cams_h)])
                e.record(st)
                if i >= warmup:
                    ev.append((s, e))
        torch.cuda.synchronize()
        return statistics.mean(s.elapsed_time(e) for s, e in ev)

    # (a) the captured graph of npvs_forward replayed per frame; (b) one npvs_forward call through
    # the C ABI per frame (host-side argument checks and launches inside the timed region)
    ms_e2e = max_over_ranks(e2e_frames(lambda c: nf.frame_from_host(g16, cam_buf, c, pvs_h), args.steps,
                                       args.warmup, fps_step), dev)

    def abi_call(c):
        cam_buf.copy_(c, non_blocking=True)
        nf.run(boxes_d, off_d, nb, cam_buf)
        pvs_h.copy_(nf.pvs, non_blocking=True)

    ms_e2e_abi = max_over_ranks(e2e_frames(abi_call, args.steps, args.warmup, max(1, fps_step // 2)), dev)
    if ops.npvs_check_status(nf.status) != 0:
        raise RuntimeError("device status set during the end-to-end frames")
    h2d = boxes_h.numel() * 4 + cams_h[0].numel()
    d2h = pvs_h.numel() * 4

    # ---- pruning (Sec. 3.2 / Sec. 5.6): every box of the scene tested against the frame's PVS
    g16.replay()
    torch.cuda.synchronize()
    vis = torch.empty(nb, dtype=torch.uint8, device=dev)
    g_pr = torch.cuda.CUDAGraph()
    ops.npvs_prune(boxes_d, off_d, cam_buf, fp.grid, wl.supersample, nf.pvs, vis)   # workspace sized, untimed
    with torch.cuda.graph(g_pr):
        ops.npvs_prune(boxes_d, off_d, cam_buf, fp.grid, wl.supersample, nf.pvs, vis)
    pr_ev = []
    for i in range(3 + 20):
        s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_.record(st)
        g_pr.replay()
        e_.record(st)
        if i >= 3:
            pr_ev.append((s_, e_))
    torch.cuda.synchronize()
    ms_prune = statistics.median(s_.elapsed_time(e_) for s_, e_ in pr_ev)
    prune = {"boxes": nb, "kept": int(vis.sum().item()), "ms": round(ms_prune, 4),
             "boxes_per_s": round(nb * 1000.0 / ms_prune, 1),
             "what": "npvs_prune of every scene box against the frame's PVS (one CUDA graph replay)"}

    # ---- roofline. The headline one is the whole frame's (the slower of its contraction FLOPs at
    # the tensor peak and its algorithmic bytes at the HBM peak, against the measured ms per frame);
    # the convolution kernels' own fraction (their algorithmic work against their summed stage
    # times) is reported beside it.
    alg = layer_algorithmic(fp, wl)
    conv_keys = [k for k in alg if k.startswith("conv:") and k in stage_ms]

    def roof_of(byts, flops, t_s):
        if flops / (tf_bf16 * 1e12) > byts / (hbm_gbs * 1e9):
            r = {"bound": "tensor", "achieved": round(flops / t_s / 1e12, 3), "peak": tf_bf16, "unit": "TFLOP/s"}
        else:
            r = {"bound": "hbm", "achieved": round(byts / t_s / 1e9, 2), "peak": hbm_gbs, "unit": "GB/s"}
        r["frac"] = round(r["achieved"] / r["peak"], 5)
        r["algorithmic_bytes"], r["algorithmic_flops"] = int(byts), int(flops)
        r["time_ms"] = round(t_s * 1e3, 4)
        r["peak_source"] = peak_src + " (MEASURED_PEAKS.json: copy GB/s, cuBLAS BF16 burst TFLOP/s)"
        return r

    frame_bytes = sum(v["bytes"] for v in alg.values())
    frame_flops = sum(v["flops"] for v in alg.values())
    roof = roof_of(frame_bytes, frame_flops, ms_frame * 1e-3)
    roof["kernel"] = "frame (every kernel of npvs_forward, one graph replay)"
    roof["traffic"], roof["traffic_frame_algorithmic_bytes"] = frame_traffic(tuned, chain_level)
    conv_roof = roof_of(sum(alg[k]["bytes"] for k in conv_keys), sum(alg[k]["flops"] for k in conv_keys),
                        sum(stage_ms[k] for k in conv_keys) * 1e-3)
    conv_roof["kernel"] = "conv (all %d layers: tcgen05 GEMM + gather-reduce kernels)" % len(conv_keys)
    conv_roof["traffic"], conv_roof["traffic_frame_algorithmic_bytes"] = frame_traffic(tuned, chain_level, True)

    line = {
        "metric": METRIC, "value": round(replica_rate(world, fps_step, ms), 3), "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
        "frames_per_step": fps_step, "ms_per_frame": round(ms_frame, 5),
        "ms_per_frame_quantiles": step_quantiles(t_bf16),
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": bench_config(world),
        "timing": {"l2": "flushed (256 MB write) before every timed frame",
                   "launch": "one CUDA graph replay of npvs_forward per frame",
                   "step": f"{fps_step} frames, each after an L2 flush and timed alone with CUDA events",
                   "timed_frames": len(t_bf16), "timed_frame_s": round(sum(t_bf16) / 1e3, 3)},
        "e2e": {"value": round(replica_rate(world, 1, ms_e2e), 3), "unit": "frames/s", "h2d_bytes_per_step": h2d * fps_step,
                "d2h_bytes_per_step": d2h * fps_step, "h2d_bytes_per_frame": h2d, "d2h_bytes_per_frame": d2h,
                "what": "pinned host boxes and camera up, PVS bits down, one graph replay of npvs_forward per frame"},
        "e2e_abi_call": {"value": round(replica_rate(world, 1, ms_e2e_abi), 3), "unit": "frames/s",
                         "what": "as e2e, with one npvs_forward call through the C ABI per frame (no graph)"},
        "gpu_launches": int(launches_timed),
        "launches_per_frame": int(launches_per_frame),
        "chain": {"level": chain_level, "layers": [wl.layers[i].name for i in P.chain_layer_indices(wl.layers, chain_level)],
                  "ms_per_frame_by_level": {str(k): round(v, 4) for k, v in chain_ms.items()},
                  "what": "layers of levels >= level run as one persistent cooperative kernel (0: every layer "
                          "its own launch); the level is chosen by timing the captured frame at each level"},
        "fp32_path": {"ms_per_frame": round(ms32, 4), "frames_per_s": round(1000.0 / ms32, 3),
                      "bf16_speedup": round(ms32 / ms_frame, 3)},
        "stage_ms": {k: round(v, 4) for k, v in sorted(stage_ms.items(), key=lambda kv: -kv[1])},
        "stage_ms_what": "stage events in a graph of the frame built entry point by entry point (no layer chain); "
                         "the events break the launch overlap, so the stages add up to more than ms_per_frame",
        "roofline": roof,
        "conv_roofline": conv_roof,
        "active_sites": [int(lv.n_rows.item()) for lv in fp.levels],
        "autotuned": {k: [tuned_label(v[0]), round(v[1], 2) if v[1] == v[1] else None] for k, v in tuned.items()},
        "tuned_source": (os.path.relpath(args.tuned, ROOT) + " (per-layer configuration autotuned earlier on a GB300)"
                         if args.tuned else "autotuned in this run"),
    }
    if clk:
        line["clocks"] = clk
    line["prune"] = prune
    if not args.no_batched:
        line["batched"] = run_batched(args, dev, net, fp.descs)
    if not args.no_highres:
        line["highres"] = run_highres(args, dev, tf_bf16, hbm_gbs)
    if not args.no_paper256:
        line["paper256"] = run_paper256(args, dev, tf_bf16, hbm_gbs)
        d1 = run_paper256_d1(args, dev, tf_bf16, hbm_gbs)
        d1["vs_interleaved"] = {"time_ratio": round(d1["ms_per_batch"] / line["paper256"]["ms_per_batch"], 2),
                                "what": "ms per frame without interleave / with d=16 (the paper's Sec. 5.4 ablation "
                                        "table: 25.4 / 10.1 ms)"}
        line["paper256_d1"] = d1
        by_d = {}
        for d in (8, 32):
            r = run_paper256_factor(args, dev, tf_bf16, hbm_gbs, d)
            line[f"paper256_d{d}"] = r
        for d in (8, 16, 32):
            r = line["paper256"] if d == 16 else line[f"paper256_d{d}"]
            by_d[str(d)] = {"ms_per_frame": r["ms_per_batch"], "peak_device_mb": r["memory_mb"]["peak_device"],
                            "active_coarse_sites": r["active_sites"][0]}
        line["paper256_by_interleave_factor"] = by_d
    if not args.no_k3:
        line["city256_k3"] = run_city256_k3(args, dev, tf_bf16, hbm_gbs)
    if not args.no_train:
        del g16, g32, g16t
        line["train"] = run_train(args, dev, flush)
        if not args.no_quality:
            line["train_quality"] = run_quality(dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        cms, cstages, G, logits, coords = cpu_oracle_frame(0)
        spent = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": round(1000.0 / cms, 5), "unit": "frames/s", "cores": os.cpu_count(),
                                "kind": "oracle", "seconds": round(spent, 1), "stage_ms": cstages,
                                "sample": "one whole frame of the FP64 / binary32-mirror oracle (froxelization of all "
                                          "65,536 columns at s=8, interleave, U-Net, de-interleave; nothing scaled)",
                                "loss_ms_not_in_frame": round(cpu_oracle_loss_ms(G, logits, coords), 1),
                                "cpu_model": cpu_model()}
        if not args.no_single_thread:
            single = cpu_oracle_single_thread(G)
            if single is not None:
                line["cpu_baseline"]["single_thread"] = {
                    "value": round(1000.0 / single[0], 5), "unit": "frames/s", "threads": 1, "stage_ms": single[1],
                    "sample": "froxelization of 2,048 random columns scaled to 65,536; the rest of the frame whole"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.grid_only:
        run_grid_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
