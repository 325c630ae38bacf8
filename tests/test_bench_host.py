"""Host logic of bench.py's multi-rank path on CPU: two gloo ranks, no GPU.

Replicas only: every rank times its own copy of the steps, the job's time is the slowest
rank's, and the value counts the units of all ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, torch.device("cpu"))
    out[rank] = ms
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == 15.0


def test_whole_job_value_counts_all_replicas():
    assert bench.whole_job_value(1, 14400, 100, 2.0) == pytest.approx(14400 * 100 / 2e-3)
    assert bench.whole_job_value(4, 14400, 100, 2.0) == pytest.approx(4 * 14400 * 100 / 2e-3)


def test_single_process_needs_no_collective():
    assert bench.max_over_ranks(3.5) == 3.5


def test_algorithmic_bytes_and_flops_of_the_paper_scale_subframe():
    """Per-launch figures the roofline divides by (one subframe, B = 12)."""
    from paper_1802_05427_gb300 import synth
    a = bench.algorithmic(synth.PAPER_SCALE, 12)
    n_h = 2 * 12 * 128 * 1200
    assert a["res_per_step"] == 14400
    assert a["ls_lmmse"]["bytes"] == 8 * n_h + 8 * 2 * 12 * 1200 + 8 * n_h + 8 * 144
    assert a["ls_lmmse"]["flops"] == 6 * n_h + 8 * 12 * n_h
    det = a["detect"]
    assert det["bytes"] == 8 * n_h + 8 * 12 * 128 * 1200 + 8 * 12 * 12 * 1200 + 12 * 12 * 1200 + 4 * 2 * 1200
    assert det["flops"] == 2400 * (8 * 128 * 78 + 8 * 12 ** 3 // 6) + 14400 * (8 * 128 * 12 + 8 * 144)


def test_roofline_rows_pick_the_binding_unit():
    """The estimator on tcgen05 is bound by HBM at B = 12 and by the FP32-accurate tensor rate
    at B = 1200 (flops / us / peak); the detector compares against HBM and FP32 FMA."""
    from paper_1802_05427_gb300 import synth
    sh = synth.PAPER_SCALE
    hbm = 6693.5
    tc_peak = bench.tf32x3_peak()[0]
    assert 300.0 < tc_peak < 340.0          # measured BF16 burst x 1.1 / 2.25 / 3
    a12 = bench.algorithmic(sh, 12)["ls_lmmse"]
    r = bench.roof_row(a12, 19.2, hbm, True)
    assert r["bound"] == "hbm" and abs(r["frac"] - a12["bytes"] / 19.2e-6 / 1e9 / hbm) < 1e-12
    a1200 = bench.algorithmic(sh, 1200)["ls_lmmse"]
    r = bench.roof_row(a1200, 258.7, hbm, True)
    assert r["bound"] == "tensor" and r["peak"] == tc_peak
    assert abs(r["frac"] - a1200["flops"] / 258.7e-6 / 1e12 / tc_peak) < 1e-12
    r = bench.roof_row(a1200, 258.7, hbm, False)  # the same work on the FP32 cores
    assert r["bound"] == "alu" and r["peak"] == bench.ALU_PEAK_TFLOPS
    r = bench.roof_row(a1200, 258.7, hbm, False, 61.5)   # against a measured FMA peak
    assert r["bound"] == "alu" and r["peak"] == 61.5
    d = bench.algorithmic(sh, 12)["detect"]
    assert bench.roof_row(d, 24.4, hbm, False)["bound"] == "hbm"


def test_timed_region_holds_exactly_the_requested_steps():
    """The timed graphs add up to --steps at any count (pipelined pieces, no serial tail)."""
    for k in (1, 3, 20, 24, 1023, 1024, 1025, 4000):
        pieces = bench.timed_pieces(k)
        assert sum(pieces) == k and all(0 < p <= bench.MAX_GRAPH_STEPS for p in pieces)
    assert bench.timed_pieces(20) == [20]
    assert bench.timed_pieces(0) == []
