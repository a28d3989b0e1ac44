"""The bench's multi-GPU path is replicas only (viewcells are independent; the path has no exchange
step): every rank times its own frames and the whole-job rate uses the slowest rank. Checked on the
CPU with two gloo ranks: the rank environment is parsed, the per-step time is the maximum over the
ranks on every rank, and the rate is world x units / time."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_env()
    dist.init_process_group("gloo", init_method="env://")
    try:
        mine = 1.5 + 2.0 * rank                      # rank 1 is the slow one
        slowest = bench.max_over_ranks(mine, "cpu")
        out[rank] = (w, r, local, slowest, bench.replica_rate(w, 1, slowest))
    finally:
        dist.destroy_process_group()


def test_replicas_time_by_slowest_rank():
    world = 2
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for rank in range(world):
        w, r, local, slowest, rate = out[rank]
        assert (w, r, local) == (world, rank, rank)
        assert slowest == pytest.approx(3.5)
        assert rate == pytest.approx(world * 1000.0 / 3.5)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.25, "cpu") == 2.25
    assert bench.replica_rate(1, 8, 4.0) == pytest.approx(2000.0)


def test_tuned_labels_and_traffic_selection():
    """The bench names the tuned forms and reports the measured frame traffic only for the chain
    level and level-0 forms it was captured with."""
    sys.path.insert(0, ROOT)
    import bench
    prod = {"tune_form": 2}
    win = {"tune_form": 1, "tune_gather": 3, "tune_max_split": 1}
    win3 = {"tune_form": 1, "tune_gather": 4}
    gat = {"tune_form": 1, "tune_gather_warps": 4}
    assert bench.tuned_label(prod) == "product"
    assert bench.tuned_label({"tune_form": 2, "tune_max_split": 8}) == "product-split"
    assert bench.tuned_label(win) == "window-nosplit"
    assert bench.tuned_label(win3) == "window3"
    assert bench.tuned_label(gat) == "gather-4w"
    assert bench.tuned_label({"tune_form": 1, "tune_gather": 4, "tune_stages": 2}) == "window3-s2"
    cfg = {"product": prod, "product-split": {"tune_form": 2, "tune_max_split": 8}, "window3": win3,
           "window3-nosplit": dict(win3, tune_max_split=1), "gather": {"tune_form": 1}}
    tuned = {k: (cfg[v], 1.0) for k, v in bench.FRAME_DRAM["forms"].items()}
    assert bench.frame_traffic(tuned, 1) == (bench.FRAME_DRAM["dram_bytes"], bench.FRAME_DRAM["algorithmic_bytes"])
    assert bench.frame_traffic(tuned, 1, True) == (bench.FRAME_DRAM["conv_dram_bytes"],
                                                   bench.FRAME_DRAM["conv_algorithmic_bytes"])
    assert bench.frame_traffic(tuned, 0) == (None, None) and bench.frame_traffic(tuned, 2) == (None, None)
    other = dict(tuned, stem=(win3, 1.0))
    assert bench.frame_traffic(other, 1) == (None, None)
    # the shipped headline configuration is the one the traffic was measured with
    import json
    shipped = {k: (v, 1.0) for k, v in json.load(open(bench.TUNED_HEADLINE)).items()}
    assert bench.frame_traffic(shipped, 1) == (bench.FRAME_DRAM["dram_bytes"], bench.FRAME_DRAM["algorithmic_bytes"])


def test_step_quantiles_nearest_rank():
    import bench
    assert bench.step_quantiles([1.0] * 98 + [2.0, 3.0]) == {"p50": 1.0, "n": 100, "p99": 2.0}
    # fewer than 100 samples: no 99th percentile, the maximum is labelled as such
    assert bench.step_quantiles(range(1, 51)) == {"p50": 25.5, "n": 50, "max": 50.0}
    assert bench.step_quantiles([]) == {"p50": None, "n": 0}


def test_frames_per_step_fills_about_a_second():
    import bench
    assert bench.frames_per_step(20, 0.5) == 100          # 20 steps x 100 frames x 0.5 ms = 1 s
    assert bench.frames_per_step(50, 30.0) == 1
    assert bench.frames_per_step(0, 0.0) >= 1
