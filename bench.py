#!/usr/bin/env python3
"""Throughput of the uplink receive path: LS -> sub-block LMMSE -> MMSE detection.

One step = one subframe of the paper-scale workload (128 antennas, 12 users, 1200
subcarriers, 2 slots x 6 data symbols, 16-QAM, sub-block B = 12 unless --subblock) through
every per-subframe stage: the fused LS + LMMSE kernel and the detection kernel.  The
LMMSE weights are plan state (built once, outside the timed region), like the paper's
precomputed weight files.  Metric: data resource elements (OFDM symbol x subcarrier, each
carrying K user symbols) detected per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl rapro|reference]

Multi-GPU (torchrun, N > 1): independent replicas, one subframe stream per rank, no
collective on the data path; value = all ranks' REs / max-over-ranks time.
--impl reference times the FP64 CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "uplink REs detected/s at 128x12, 1200 sc (FP32 vs BF16-TC); % roofline"
UNIT = "REs/s"
N_SETS = 8                   # resident input subframes rotated through (> L2 in total)
GRAPH_STEPS = 3 * N_SETS     # steps per captured CUDA graph
IN_FLIGHT = 4                # subframes in flight: consecutive steps rotate over 4 streams
MAX_GRAPH_STEPS = 1024       # steps per graph of the timed region
L2_BYTES = 129 * 2 ** 20
# FP32 FMA lanes x 2 flop x max SM clock: context, and the fallback when the measured rate
# (rapro_measure_ffma_peak, taken by every run) is not available
ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=64)
    ap.add_argument("--impl", choices=["rapro", "reference"], default="rapro")
    ap.add_argument("--subblock", type=int, default=12)
    ap.add_argument("--snr", type=float, default=10.0)
    ap.add_argument("--no-sweep", action="store_true", help="skip every extra section")
    ap.add_argument("--sections", default="sweep,precision,differentiable,hetero,comb,batch64",
                    help="extra sections after the headline line's measurement (comma list)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=100)
    return ap.parse_args()


def workload(args):
    from paper_1802_05427_gb300 import synth
    sh = synth.SubframeShape(**{**synth.PAPER_SCALE.__dict__, "snr_db": args.snr})
    desc = (f"paper-scale plain FP32 receive: M={sh.M} antennas, K={sh.K} users, {sh.n_sc} subcarriers "
            f"(FFT {sh.n_fft}), 1 subframe = {sh.n_slots} slots x {sh.n_data_per_slot} data symbols, "
            f"{1 << sh.qam_bits}-QAM, {sh.n_taps}-tap exponential PDP (tau {sh.tau_rms:g}), SNR {sh.snr_db:g} dB, "
            f"sub-block B={args.subblock}")
    return sh, desc


def algorithmic(sh, B):
    """Algorithmic bytes and flops per launch (one subframe) of each kernel."""
    T, K, M, N, D = sh.n_slots, sh.K, sh.M, sh.n_sc, sh.n_data_per_slot
    c = 8
    n_h = T * K * M * N
    tail = N % B
    w_bytes = c * (B * B + tail * tail)
    flops_lmmse = 8 * n_h * B if tail == 0 else 8 * T * K * M * ((N - tail) * B + tail * tail)
    est = dict(bytes=c * n_h + c * T * K * N + c * n_h + w_bytes, flops=6 * n_h + flops_lmmse)
    res = T * D * N
    det_bytes = c * n_h + c * T * D * M * N + c * T * D * K * N + T * D * K * N + 4 * T * N
    det_flops = (T * N * (8 * M * K * (K + 1) // 2 + 8 * K ** 3 // 6)) + res * (8 * M * K + 8 * K * K)
    # the whole path as one algorithm (Eq. 9, 12, 20-22): inputs once, results once, h on chip
    path_bytes = (c * n_h + c * T * K * N + c * T * D * M * N + w_bytes + c * T * D * K * N + T * D * K * N
                  + 4 * T * N)
    path = dict(bytes=path_bytes, flops=est["flops"] + det_flops)
    return dict(ls_lmmse=est, detect=dict(bytes=det_bytes, flops=det_flops), path=path, res_per_step=res)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def tf32x3_peak():
    """Peak rate of FP32-accurate algorithmic flops on the tensor cores: the TF32 dense rate
    (measured BF16 burst x the nominal TF32 / BF16 ratio 1.1 / 2.25) over the 3 TF32 passes."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16, kind = float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        bf16, kind = 1900.0, "fallback"
    return bf16 * 1.1 / 2.25 / 3.0, f"{kind} BF16 {bf16:g} TFLOP/s x 1.1/2.25 (TF32) / 3 passes"


def roof_row(a, us, hbm, on_tc, alu_peak=None):
    """One kernel against its roofline: the larger of its algorithmic bytes over the HBM
    copy rate and its flops over the rate of the unit that does them (FP32 FMA at alu_peak
    TFLOP/s, measured, else the derived figure; or the FP32-accurate tensor rate when on_tc);
    achieved = the same quantity over the measured launch time us (microseconds)."""
    tc_peak, tc_src = tf32x3_peak()
    cpeak = tc_peak if on_tc else (alu_peak or ALU_PEAK_TFLOPS)
    if a["bytes"] / (hbm * 1e9) >= a["flops"] / (cpeak * 1e12):
        ach, peak, unit, bound = a["bytes"] / (us * 1e-6) / 1e9, hbm, "GB/s", "hbm"
    else:
        ach, peak, unit, bound = a["flops"] / (us * 1e-6) / 1e12, cpeak, "TFLOP/s", "tensor" if on_tc else "alu"
    row = dict(bound=bound, achieved=ach, peak=peak, unit=unit, frac=ach / peak, us_per_launch=us,
               alg_bytes=a["bytes"], alg_flops=a["flops"])
    if on_tc:
        row["tensor_peak_source"] = tc_src
    return row


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1802_05427_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h", ".cpp")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it matches these kernels."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except Exception:
        return None
    if t.get("source_hash") != kernel_source_hash():
        return None
    v = t.get("kernels", {}).get(kernel)
    return None if v is None else float(v)


# ------------------------------------------------- batched heterogeneous workload
def hetero_batch(dev, n_jobs=512, seed=0x18020542 + 3, bf16=False):
    """512 jobs: M ~ U{32,64,128,256}, K ~ U{4,8,12,16}, n_sc ~ U{72,300,600,1200} (FFT the next of
    128/512/1024/2048), 2/4/6-bit QAM, SNR ~ U[0,25] dB, tau ~ U[2,12], B ~ U{12,48}; inputs are
    seeded device Gaussians with unit-modulus pilots (the kernels' work does not depend on the
    values).  One CUDA graph of rapro_receive_batch over all jobs, 8 streams vs 1 stream, and
    after rapro_plan_tune on every plan.  bf16: each job's filter in the BF16 form where its
    shape allows it (B dividing n_sc), else FP32."""
    import torch
    from paper_1802_05427_gb300 import rapro as R
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    fft_of = {72: 128, 300: 512, 600: 1024, 1200: 2048}
    jobs, res, n_bf16 = [], 0, 0
    for _ in range(n_jobs):
        M = int(rng.choice([32, 64, 128, 256]))
        K = int(rng.choice([4, 8, 12, 16]))
        N = int(rng.choice([72, 300, 600, 1200]))
        q = int(rng.choice([2, 4, 6]))
        snr = float(rng.uniform(0.0, 25.0))
        tau = float(rng.uniform(2.0, 12.0))
        B = int(rng.choice([12, 48]))
        p = R.make_params(M=M, K=K, n_sc=N, n_fft=fft_of[N], subblock=B, sigma2=10 ** (-snr / 10), qam_bits=q,
                          n_taps=16, tau_rms=tau)
        if bf16:
            p.precision = R.RAPRO_PREC_BF16
            if R.rapro_params_validate(p) != R.RAPRO_OK:
                p.precision = R.RAPRO_PREC_FP32
            n_bf16 += p.precision == R.RAPRO_PREC_BF16
        pl = R.Plan(p)
        if p.precision != R.RAPRO_PREC_FP32:
            # the batch workload asks for BF16 filtering; its detectors stay FP32
            R.rapro_plan_set_detector_form(pl, R.RAPRO_DET_FP32)
        s = pl.shapes()

        def cn(shape):
            return torch.complex(torch.randn(shape, generator=gen, device=dev),
                                 torch.randn(shape, generator=gen, device=dev)).contiguous()
        th = torch.rand(s["pilots"], generator=gen, device=dev) * (2 * np.pi)
        jobs.append(dict(plan=pl, y_pilot=cn(s["y_pilot"]), pilots=torch.polar(torch.ones_like(th), th).contiguous(),
                         y_data=cn(s["y_data"]), x_eq=torch.empty(s["x_eq"], dtype=torch.complex64, device=dev),
                         labels=torch.empty(s["labels"], dtype=torch.uint8, device=dev)))
        res += pl.T * pl.D * N
    torch.cuda.synchronize()

    def timed(n_streams, reps=5):
        batch = R.Batch(n_streams)
        R.rapro_receive_batch(batch, jobs)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        st = torch.cuda.Stream()
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            with torch.cuda.graph(g, stream=st):
                R.rapro_receive_batch(batch, jobs, stream=st)
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        batch.close()
        return e0.elapsed_time(e1) / reps

    ms8, ms1 = timed(8), (timed(1) if not bf16 else 0.0)
    t0 = time.time()
    for j in jobs:
        s = j["plan"].shapes()
        h = torch.empty(s["h"], dtype=torch.complex64, device=dev)
        R.rapro_plan_tune(j["plan"], j["y_pilot"], j["pilots"], j["y_data"], h, j["x_eq"])
    tune_s = time.time() - t0
    ms8t = timed(8)
    counts = {}
    for j in jobs:
        ev = R.rapro_plan_variant(j["plan"])[0]
        counts[str(ev)] = counts.get(str(ev), 0) + 1
    for j in jobs:
        assert j["plan"].device_status() == 0
        j["plan"].close()
    if bf16:
        return {"jobs": n_jobs, "bf16_jobs": int(n_bf16), "ms_per_batch_8_streams": ms8,
                "res_per_s_8_streams": res / (ms8 * 1e-3), "res_per_s_8_streams_tuned": res / (ms8t * 1e-3)}
    return {"jobs": n_jobs, "res_per_batch": res, "ms_per_batch_8_streams": ms8, "ms_per_batch_1_stream": ms1,
            "res_per_s_8_streams": res / (ms8 * 1e-3), "res_per_s_1_stream": res / (ms1 * 1e-3),
            "res_per_s_8_streams_tuned": res / (ms8t * 1e-3), "tune_seconds": tune_s,
            "tuned_estimator_kernels": counts,
            "inputs": "seeded device Gaussians (unit-modulus pilots), one CUDA graph per batch"}


def measure_ffma(R, dev, trips=50000, runs=5):
    """FP32 FMA peak of this GPU: the library's FMA-chain probe (full occupancy, 8
    independent chains per thread), best of `runs` launches, with the SM clock sampled
    during them; flop_per_clk_per_sm checks the figure against 2 x 128 lanes."""
    import torch
    clocks = ClockSampler(gpu_id_for(dev))
    clocks.start()
    time.sleep(0.3)
    R.rapro_measure_ffma_peak(2000)
    t0 = time.time()
    got = [R.rapro_measure_ffma_peak(trips) for _ in range(runs)]
    t1 = time.time()
    time.sleep(0.2)
    clocks.stop()
    clk = clocks.summary(t0, t1, "the probe's launches")
    tf = max(g[0] for g in got)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = {"tflops": tf, "tflops_median": statistics.median(g[0] for g in got),
           "ms_per_launch": statistics.median(g[1] for g in got), "sms": sms, "clocks": clk,
           "derived_at_max_clock_tflops": sms * 128 * 2 * 2.070e9 / 1e12,
           "source": "rapro_measure_ffma_peak: 8 CTAs x 256 threads per SM, 8 independent FMA chains per "
                     f"thread, {16 * trips} rounds, best of {runs} (CUDA events)"}
    if clk.get("sm_mhz"):
        out["flop_per_clk_per_sm"] = tf * 1e12 / (sms * clk["sm_mhz"] * 1e6)
    return out


def precision_accuracy(R, synth, dev, B, n_sub=20):
    """NMSE of h and EVM of x~ over n_sub paper-scale subframes (64-QAM, 25 dB) for the FP32,
    BF16 and FP16 forms, each against the true channel and transmitted symbols."""
    import torch
    sh = synth.SubframeShape(**{**synth.PAPER_SCALE.__dict__, "snr_db": 25.0, "qam_bits": 6})
    forms = {"fp32": R.RAPRO_PREC_FP32, "bf16_tc": R.RAPRO_PREC_BF16, "fp16_tc": R.RAPRO_PREC_FP16}
    plans = {}
    for name, pv in forms.items():
        plans[name] = R.Plan(R.make_params(M=sh.M, K=sh.K, n_sc=sh.n_sc, n_fft=sh.n_fft, subblock=B,
                                           sigma2=sh.sigma2, qam_bits=sh.qam_bits, n_taps=sh.n_taps,
                                           tau_rms=sh.tau_rms, precision=pv))
    s = plans["fp32"].shapes()
    acc = {name: [0.0, 0.0] for name in forms}
    pow_h = pow_x = 0.0
    x = torch.empty(s["x_eq"], dtype=torch.complex64, device=dev)
    h = torch.empty(s["h"], dtype=torch.complex64, device=dev)
    for i in range(n_sub):
        sf = synth.make_subframe(sh, seed=synth.SEED_BASE + 9000 + i)
        ins = [torch.from_numpy(synth.as_c64(sf[k])).to(dev) for k in ("y_pilot", "pilots", "y_data")]
        H = np.transpose(sf["H"], (1, 0, 2))[None]
        pow_h += sh.n_slots * float(np.sum(np.abs(H) ** 2))
        pow_x += float(np.sum(np.abs(sf["x"]) ** 2))
        for name, pl in plans.items():
            R.rapro_receive_subframe(pl, *ins, x, h_out=h)
            torch.cuda.synchronize()
            acc[name][0] += float(np.sum(np.abs(h.cpu().numpy() - H) ** 2))
            acc[name][1] += float(np.sum(np.abs(x.cpu().numpy() - sf["x"]) ** 2))
    out = {"workload": f"{sh.M}x{sh.K}, {sh.n_sc} sc, {n_sub} subframes, 64-QAM, 25 dB, B = {B}",
           "reference": "true channel and transmitted symbols of the generator"}
    db = lambda v: 10.0 * np.log10(v)
    for name, pl in plans.items():
        assert pl.device_status() == 0
        nmse, evm = db(acc[name][0] / pow_h), db(acc[name][1] / pow_x)
        out[name] = {"nmse_db": nmse, "evm_db": evm, "evm_pct": 100.0 * np.sqrt(acc[name][1] / pow_x)}
        pl.close()
    for name in ("bf16_tc", "fp16_tc"):
        out[name]["nmse_minus_fp32_db"] = out[name]["nmse_db"] - out["fp32"]["nmse_db"]
        out[name]["evm_minus_fp32_db"] = out[name]["evm_db"] - out["fp32"]["evm_db"]
    return out


# ------------------------------------------------------------ multi-rank
def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest of every rank's value (a timed region ends when the slowest rank does)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def timed_pieces(steps: int) -> list:
    """Step counts of the graphs that make up a timed region of `steps` steps."""
    full, rest = divmod(max(int(steps), 0), MAX_GRAPH_STEPS)
    return [MAX_GRAPH_STEPS] * full + ([rest] if rest else [])


def whole_job_value(world: int, units_per_step: int, steps: int, ms: float) -> float:
    """Units all ranks processed per second: every rank runs its own replica of the steps."""
    return world * units_per_step * steps / (ms * 1e-3)


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1, window):
        sm, mx, reasons = [], [], set()
        for ts, line in self.rows:
            if not (t0 <= ts <= t1):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                 parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "window": window}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "window": window}


def gpu_id_for(dev):
    """Something nvidia-smi -i accepts for this CUDA device (PCI id, else the visible id)."""
    import torch
    try:
        p = torch.cuda.get_device_properties(dev)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    if ids and dev.index is not None and dev.index < len(ids):
        return ids[dev.index].strip()
    return None


# ------------------------------------------------------------ CPU oracle
_JOB_INPUTS = {}


def _oracle_job(job):
    """Worker: time the FP64 oracle on `n_sub` subframes restricted to `n_sc` subcarriers.

    Inputs are drawn once per (seed, n_sc) and kept in the worker, outside the timing."""
    import numpy as np
    from oracle import rapro_oracle as O
    from paper_1802_05427_gb300 import synth
    shape_kw, B, n_sc, n_sub, seed = job
    sh = synth.SubframeShape(**shape_kw)
    key = (seed, n_sc)
    if key not in _JOB_INPUTS:
        _JOB_INPUTS.clear()
        sf = synth.make_subframe(sh, seed=seed)
        _JOB_INPUTS[key] = {k: np.ascontiguousarray(synth.as_c64(sf[k])[..., :n_sc].astype(np.complex128))
                            for k in ("y_pilot", "pilots", "y_data")}
    c = _JOB_INPUTS[key]
    r = O.make_r("exp", n_taps=sh.n_taps, tau_rms=sh.tau_rms, n_fft=sh.n_fft)
    t0 = time.perf_counter()
    for _ in range(n_sub):
        O.receive_subframe(c["y_pilot"], c["pilots"], c["y_data"], B=B, sigma2=sh.sigma2, r=r,
                           n_data_per_slot=sh.n_data_per_slot, q=sh.qam_bits)
    dt = time.perf_counter() - t0
    return n_sub * sh.n_slots * sh.n_data_per_slot * n_sc, dt


def oracle_pool(n_workers):
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"          # one BLAS thread per worker process
    return mp.get_context("spawn").Pool(n_workers)


def cpu_baseline(sh, B, target_s=12.0):
    n = os.cpu_count() or 1
    shape_kw = dict(sh.__dict__)
    with oracle_pool(n) as pool:
        res, dt = pool.map(_oracle_job, [(shape_kw, B, sh.n_sc, 1, 7000 + i) for i in range(n)])[0]
        per_sub = max(dt, 1e-3)
        n_sub = max(1, int(target_s / per_sub))
        out = pool.map(_oracle_job, [(shape_kw, B, sh.n_sc, n_sub, 7100 + i) for i in range(n)])
        # one process alone: the single-core rate
        res1, dt1 = pool.map(_oracle_job, [(shape_kw, B, sh.n_sc, 1, 7200)])[0]
    res_total = sum(r for r, _ in out)
    t = max(d for _, d in out)
    return {"value": res_total / t, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{n} processes x {n_sub} full subframes each (1 BLAS thread per process), "
                      f"{res_total} REs in {t:.1f} s",
            "single_core": {"value": res1 / max(dt1, 1e-9), "unit": UNIT,
                            "sample": f"1 process, 1 BLAS thread, 1 full subframe ({res1} REs in {dt1:.2f} s)"}}


# ----------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sh, desc = workload(args)
    B = args.subblock
    n = os.cpu_count() or 1
    shape_kw = dict(sh.__dict__)
    budget_s = 150.0
    with oracle_pool(n) as pool:
        _, dt = pool.map(_oracle_job, [(shape_kw, B, sh.n_sc, 1, 8000 + i) for i in range(n)])[0]
        per_sc = dt / sh.n_sc
        steps_total = args.steps + args.warmup
        n_sc = max(B, min(sh.n_sc, int(budget_s / max(steps_total, 1) / per_sc) // B * B))
        jobs = [(shape_kw, B, n_sc, 1, 8100 + i) for i in range(n)]
        for _ in range(args.warmup):
            pool.map(_oracle_job, jobs)
        t0 = time.perf_counter()
        res = 0
        for _ in range(args.steps):
            res += sum(r for r, _ in pool.map(_oracle_job, jobs))
        wall = time.perf_counter() - t0
    value = res / wall
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "subblock": B, "snr_db": sh.snr_db},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle",
                             "sample": f"each step: {n} processes x 1 "
                                       + ("full subframe" if n_sc == sh.n_sc else
                                          f"subframe restricted to the first {n_sc} subcarriers")
                                       + f" ({n_sc // B} blocks of {B}); inputs drawn once "
                                       "per worker outside the timing"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_rapro(args):
    import numpy as np
    import torch

    from paper_1802_05427_gb300 import _build, synth
    from paper_1802_05427_gb300 import rapro as R

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # CPU baseline first: its spawn pool must not fork a CUDA-initialised process.
    sh, desc = workload(args)
    B = args.subblock
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sh, B)

    if rank == 0:
        _build.build()
    if dist:
        dist.barrier()
    R.lib()

    def want(section):
        return not args.no_sweep and section in args.sections.split(",")

    alg = algorithmic(sh, B)
    res_per_step = alg["res_per_step"]
    params = R.make_params(M=sh.M, K=sh.K, n_sc=sh.n_sc, n_fft=sh.n_fft, subblock=B, sigma2=sh.sigma2,
                           qam_bits=sh.qam_bits, n_taps=sh.n_taps, tau_rms=sh.tau_rms)
    plan = R.Plan(params)
    s = plan.shapes()
    sets = []
    for i in range(N_SETS):
        sf = synth.make_subframe(sh, seed=synth.SEED_BASE + 1000 * rank + i)
        sets.append({k: torch.from_numpy(synth.as_c64(sf[k])).to(dev) for k in ("y_pilot", "pilots", "y_data")})
    in_bytes = sum(t.numel() * t.element_size() for t in sets[0].values())
    # one output set per pipeline: consecutive subframes alternate between IN_FLIGHT streams
    outs = [dict(h=torch.empty(s["h"], dtype=torch.complex64, device=dev),
                 x=torch.empty(s["x_eq"], dtype=torch.complex64, device=dev),
                 lab=torch.empty(s["labels"], dtype=torch.uint8, device=dev),
                 info=torch.empty(s["info"], dtype=torch.int32, device=dev)) for _ in range(IN_FLIGHT)]
    h, x, lab, info = outs[0]["h"], outs[0]["x"], outs[0]["lab"], outs[0]["info"]

    def step(i, which=("est", "det"), stream=None):
        d, o = sets[i % N_SETS], outs[i % IN_FLIGHT]
        if "est" in which:
            R.rapro_ce_ls_lmmse(plan, d["y_pilot"], d["pilots"], o["h"], stream=stream)
        if "det" in which:
            R.rapro_mmse_detect(plan, o["h"], d["y_data"], o["x"], o["lab"], None, o["info"], stream=stream)

    # eager warm-up (also compiles nothing: kernels are prebuilt)
    for i in range(max(args.warmup, 3)):
        step(i)
    torch.cuda.synchronize()

    def capture(which, n, start=0, pipelines=1):
        """Graph of steps start..start+n-1; step i runs on pipeline stream i % pipelines."""
        g = torch.cuda.CUDAGraph()
        st = torch.cuda.Stream()
        side = [torch.cuda.Stream() for _ in range(pipelines)]
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            with torch.cuda.graph(g, stream=st):
                fork = torch.cuda.Event()
                fork.record(st)
                for q in side:
                    q.wait_event(fork)
                for i in range(start, start + n):
                    step(i, which, stream=side[i % pipelines])
                for q in side:
                    join = torch.cuda.Event()
                    join.record(q)
                    st.wait_event(join)
        torch.cuda.synchronize()
        return g

    # The timed region replays graphs holding exactly --steps steps (in pieces of at most
    # MAX_GRAPH_STEPS), each rotating consecutive steps over IN_FLIGHT streams: the region is
    # the pipelined path at any step count, with one pipeline fill and drain per piece.
    g_full = capture(("est", "det"), GRAPH_STEPS, pipelines=IN_FLIGHT)       # warm-up and soak
    pieces = timed_pieces(args.steps)
    g_timed = {n: capture(("est", "det"), n, pipelines=IN_FLIGHT) for n in sorted(set(pieces))}
    for g in g_timed.values():            # first replays (graph upload) stay out of the region
        g.replay()
    torch.cuda.synchronize()
    g_est = capture(("est",), GRAPH_STEPS)
    g_det = capture(("det",), GRAPH_STEPS)

    def run_steps(k):
        for n in timed_pieces(k):
            g_timed[n].replay()

    clocks = ClockSampler(gpu_id_for(dev))
    clocks.start()
    time.sleep(0.3)
    # sustained load before the timed region so the clock samples see a loaded GPU
    t_soak = time.time()
    while time.time() - t_soak < 1.5:
        for _ in range(16):
            g_full.replay()
        torch.cuda.synchronize()

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_host0 = time.time()
    ev0.record()
    run_steps(args.steps)
    ev1.record()
    torch.cuda.synchronize()
    t_host1 = time.time()
    if dist:
        dist.barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    time.sleep(0.25)
    clocks.stop()
    window = "1.5 s of sustained graph replays right before the timed region, plus the timed region"
    clk = clocks.summary(t_soak, t_host1 + 0.2, window)

    # per-kernel average launch durations: graphs of GRAPH_STEPS launches of one kernel
    def time_graph(g, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / (reps * GRAPH_STEPS)   # us per launch

    reps = max(16, min(500, args.steps // GRAPH_STEPS))
    us_est, us_det = time_graph(g_est, reps), time_graph(g_det, reps)
    assert plan.device_status() == 0, "device status reports a timeout"
    ffma = measure_ffma(R, dev)

    # end to end through the user API with pinned host buffers (copies inside the region)
    rx = R.Receiver(params, device=local)
    host_sets = []
    for i in range(2):
        sf = synth.make_subframe(sh, seed=synth.SEED_BASE + 500 + i)
        host_sets.append({k: torch.from_numpy(synth.as_c64(sf[k])).pin_memory() for k in ("y_pilot", "pilots", "y_data")})
    # one pinned output set per Receiver slot: a subframe's results land while the next one runs
    outs_h = [(torch.empty(s["x_eq"], dtype=torch.complex64).pin_memory(),
               torch.empty(s["labels"], dtype=torch.uint8).pin_memory()) for _ in range(len(rx.slots))]
    for i in range(3):
        d = host_sets[i % 2]
        rx.receive_host(d["y_pilot"], d["pilots"], d["y_data"], *outs_h[i % len(outs_h)])
    rx.join()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    rx.fork()
    for i in range(args.e2e_steps):
        d = host_sets[i % 2]
        rx.receive_host(d["y_pilot"], d["pilots"], d["y_data"], *outs_h[i % len(outs_h)])
    rx.join()
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    h2d = sum(t.numel() * t.element_size() for t in host_sets[0].values())
    d2h = outs_h[0][0].numel() * outs_h[0][0].element_size() + outs_h[0][1].numel()

    # sub-block sweep of the same workload (B = 12, 48, 100, 1200), graph replays
    sweep = {}
    if want("sweep") and rank == 0 and world == 1:
        for Bs in (12, 48, 100, 1200):
            ps = R.make_params(M=sh.M, K=sh.K, n_sc=sh.n_sc, n_fft=sh.n_fft, subblock=Bs, sigma2=sh.sigma2,
                               qam_bits=sh.qam_bits, n_taps=sh.n_taps, tau_rms=sh.tau_rms)
            with R.Plan(ps) as pl2:
                def step2(i, stream=None):
                    d, o = sets[i % N_SETS], outs[i % IN_FLIGHT]
                    R.rapro_ce_ls_lmmse(pl2, d["y_pilot"], d["pilots"], o["h"], stream=stream)
                    R.rapro_mmse_detect(pl2, o["h"], d["y_data"], o["x"], o["lab"], None, o["info"], stream=stream)
                for i in range(3):
                    step2(i)
                # the same pipelining as the headline: consecutive steps rotate over IN_FLIGHT streams
                g = torch.cuda.CUDAGraph()
                st = torch.cuda.Stream()
                side = [torch.cuda.Stream() for _ in range(IN_FLIGHT)]
                st.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(st):
                    with torch.cuda.graph(g, stream=st):
                        fork = torch.cuda.Event()
                        fork.record(st)
                        for q in side:
                            q.wait_event(fork)
                        for i in range(GRAPH_STEPS):
                            step2(i, stream=side[i % IN_FLIGHT])
                        for q in side:
                            join = torch.cuda.Event()
                            join.record(q)
                            st.wait_event(join)
                torch.cuda.synchronize()
                r2 = 64 if Bs < 1200 else 4
                e0.record()
                for _ in range(r2):
                    g.replay()
                e1.record()
                torch.cuda.synchronize()
                sweep[str(Bs)] = res_per_step * r2 * GRAPH_STEPS / (e0.elapsed_time(e1) * 1e-3)

    # precision forms: the sub-block filter as one BF16 or FP16 pass on the tensor cores.  The
    # detector of such a plan keeps its FP64-fallback list in the plan, so each pipeline
    # stream gets a plan of its own.
    prec = {}
    if want("precision") and rank == 0 and world == 1 and B % 2 == 0 and B <= 16 and sh.n_sc % B == 0:
        forms = [("bf16_tc", R.RAPRO_PREC_BF16, B), ("fp16_tc", R.RAPRO_PREC_FP16, B)]
        if want("sweep"):                  # the sub-block sweep of the precision forms
            forms += [(f"{n}_B{Bs}", pv, Bs) for Bs in (48, 100, 1200)
                      for n, pv in (("bf16_tc", R.RAPRO_PREC_BF16), ("fp16_tc", R.RAPRO_PREC_FP16))]
        for name, pv, Bp in forms:
            pb = R.make_params(M=sh.M, K=sh.K, n_sc=sh.n_sc, n_fft=sh.n_fft, subblock=Bp, sigma2=sh.sigma2,
                               qam_bits=sh.qam_bits, n_taps=sh.n_taps, tau_rms=sh.tau_rms, precision=pv)
            plbs = [R.Plan(pb) for _ in range(IN_FLIGHT)]

            def bstep(i, which="full", stream=None):
                d, o, plb = sets[i % N_SETS], outs[i % IN_FLIGHT], plbs[i % IN_FLIGHT]
                if which != "det":
                    R.rapro_ce_ls_lmmse(plb, d["y_pilot"], d["pilots"], o["h"], stream=stream)
                if which != "est":
                    R.rapro_mmse_detect(plb, o["h"], d["y_data"], o["x"], o["lab"], None, o["info"], stream=stream)
            for i in range(3):
                bstep(i)
            torch.cuda.synchronize()
            gb = []
            for which, pipes in (("full", IN_FLIGHT), ("est", 1), ("det", 1)):
                g = torch.cuda.CUDAGraph()
                st = torch.cuda.Stream()
                side = [torch.cuda.Stream() for _ in range(pipes)]
                st.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(st):
                    with torch.cuda.graph(g, stream=st):
                        fork = torch.cuda.Event()
                        fork.record(st)
                        for q in side:
                            q.wait_event(fork)
                        for i in range(GRAPH_STEPS):
                            bstep(i, which, stream=side[i % pipes])
                        for q in side:
                            join = torch.cuda.Event()
                            join.record(q)
                            st.wait_event(join)
                torch.cuda.synchronize()
                gb.append(g)
            reps_b = 64 if Bp < 1200 else 4
            us_b_full, us_b_est = time_graph(gb[0], reps_b), time_graph(gb[1], reps_b)
            us_b_det = time_graph(gb[2], reps_b)
            prec[name] = {"res_per_s": res_per_step / (us_b_full * 1e-6), "estimator_us": us_b_est,
                          "detector_us": us_b_det,
                          "detector": "tensor-core Gram of 16-bit operands + FP32 Cholesky + one FP32 refinement step"}
            if Bp == B:
                # the same plans with the FP32 detector (RAPRO_DET_FP32): the 16-bit filter alone
                for plb in plbs:
                    R.rapro_plan_set_detector_form(plb, R.RAPRO_DET_FP32)
                gb[0].replay()
                torch.cuda.synchronize()
                for i in range(3):
                    bstep(i)
                torch.cuda.synchronize()
                g32 = []
                for which, pipes in (("full", IN_FLIGHT), ("det", 1)):
                    g = torch.cuda.CUDAGraph()
                    st = torch.cuda.Stream()
                    side = [torch.cuda.Stream() for _ in range(pipes)]
                    st.wait_stream(torch.cuda.current_stream())
                    with torch.cuda.stream(st):
                        with torch.cuda.graph(g, stream=st):
                            fork = torch.cuda.Event()
                            fork.record(st)
                            for q in side:
                                q.wait_event(fork)
                            for i in range(GRAPH_STEPS):
                                bstep(i, which, stream=side[i % pipes])
                            for q in side:
                                join = torch.cuda.Event()
                                join.record(q)
                                st.wait_event(join)
                    torch.cuda.synchronize()
                    g32.append(g)
                prec[name]["fp32_detector"] = {"res_per_s": res_per_step / (time_graph(g32[0], reps_b) * 1e-6),
                                               "detector_us": time_graph(g32[1], reps_b),
                                               "detector": "RAPRO_DET_FP32: FP32 Gram, FP64 fallback"}
            if Bp == B:
                prec[name]["estimator_hbm_frac"] = alg["ls_lmmse"]["bytes"] / (us_b_est * 1e-6) / (peaks()[0] * 1e9)
            for plb in plbs:
                assert plb.device_status() == 0
                plb.close()

    # The precision workload (128 x 12 x 1200, 20 subframes, 64-QAM, 25 dB, B = 12): channel
    # NMSE and EVM of the equalised symbols of the FP32 path and of each 16-bit form, against
    # the generator's true channel and transmitted symbols (the tests tie the FP32 path to the
    # FP64 oracle at 1e-5, so the FP32 figures stand for the oracle's).
    if want("precision") and rank == 0 and world == 1 and B % 2 == 0 and B <= 16 and sh.n_sc % B == 0:
        prec["accuracy_20_subframes_64qam_25db"] = precision_accuracy(R, synth, dev, B)

    # differentiable receive: forward + adjoint per subframe, and an Adam fit of (sigma2, tau)
    diff = {}
    if want("differentiable") and rank == 0 and world == 1:
        from paper_1802_05427_gb300 import autograd as AG
        shd = synth.SubframeShape(**{**synth.PAPER_SCALE.__dict__, "K": 16, "snr_db": 15.0, "tau_rms": 6.0})
        batch = []
        for i in range(8):
            sf = synth.make_subframe(shd, seed=synth.SEED_BASE + 3000 + i)
            batch.append({k: torch.from_numpy(synth.as_c64(sf[k])).to(dev) for k in ("y_pilot", "pilots", "y_data")})
            batch[-1]["x_ref"] = torch.from_numpy(synth.as_c64(sf["x"])).to(dev)
        dshape = dict(M=shd.M, K=shd.K, n_sc=shd.n_sc, n_fft=shd.n_fft, subblock=12, qam_bits=shd.qam_bits,
                      n_taps=shd.n_taps)
        pd = R.make_params(**dshape, sigma2=shd.sigma2, tau_rms=shd.tau_rms)
        with R.Plan(pd) as pld:
            sd = pld.shapes()
            hd = torch.empty(sd["h"], dtype=torch.complex64, device=dev)
            ghd = torch.empty_like(hd)
            xd = torch.empty(sd["x_eq"], dtype=torch.complex64, device=dev)
            scd = torch.empty(2, dtype=torch.float32, device=dev)
            gw = torch.empty((12, 12), dtype=torch.complex64, device=dev)

            def fb(i):
                d = batch[i % len(batch)]
                R.rapro_receive_subframe(pld, d["y_pilot"], d["pilots"], d["y_data"], xd, h_out=hd)
                R.rapro_mse_backward(pld, d["y_pilot"], d["pilots"], d["y_data"], hd, xd, d["x_ref"], ghd, scd, gw)
            for i in range(3):
                fb(i)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for i in range(32):
                fb(i)
            e1.record()
            torch.cuda.synchronize()
            diff["fwd_bwd_us_per_subframe"] = e0.elapsed_time(e1) * 1e3 / 32
        theta0 = torch.tensor([2 * shd.sigma2, 2 * shd.tau_rms], dtype=torch.float64)
        log_t = torch.log(theta0).clone().requires_grad_(True)
        opt = torch.optim.Adam([log_t], lr=0.05)
        t_fit = time.time()
        l0 = None
        for it in range(200):
            opt.zero_grad()
            l = AG.symbol_mse(torch.exp(log_t), batch, dshape)
            l0 = float(l.detach()) if l0 is None else l0
            l.backward()
            opt.step()
        fit = torch.exp(log_t.detach())
        diff.update({"workload": f"{shd.M}x{shd.K}, {shd.n_sc} sc, 8 subframes, 16-QAM, 15 dB, tau 6, B = 12",
                     "adam_steps": 200, "fit_seconds": time.time() - t_fit,
                     "theta_true": [shd.sigma2, shd.tau_rms], "theta_init": theta0.tolist(), "theta_fit": fit.tolist(),
                     "loss_init": l0, "loss_fit": float(AG.symbol_mse(fit, batch, dshape)),
                     "loss_true": float(AG.symbol_mse(torch.tensor([shd.sigma2, shd.tau_rms], dtype=torch.float64),
                                                      batch, dshape))})

    # batched heterogeneous receive: 512 subframes of uneven shapes in one call / one graph
    hetero = {}
    if want("hetero") and rank == 0 and world == 1:
        hetero = hetero_batch(dev)
        hetero["bf16_filter_where_allowed"] = hetero_batch(dev, bf16=True)

    # 64 paper-scale subframes in one rapro_receive_batch call (one plan, 8 library streams,
    # one CUDA graph per batch; the inputs rotate over the resident sets, every job has its
    # own outputs)
    batch64 = {}
    if want("batch64") and rank == 0 and world == 1:
        n64 = 64
        jobs64 = [dict(plan=plan, y_pilot=sets[i % N_SETS]["y_pilot"], pilots=sets[i % N_SETS]["pilots"],
                       y_data=sets[i % N_SETS]["y_data"], h_out=torch.empty(s["h"], dtype=torch.complex64, device=dev),
                       x_eq=torch.empty(s["x_eq"], dtype=torch.complex64, device=dev),
                       labels=torch.empty(s["labels"], dtype=torch.uint8, device=dev)) for i in range(n64)]
        b64 = R.Batch(8)
        R.rapro_receive_batch(b64, jobs64)
        torch.cuda.synchronize()
        g64 = torch.cuda.CUDAGraph()
        st64 = torch.cuda.Stream()
        st64.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st64):
            with torch.cuda.graph(g64, stream=st64):
                R.rapro_receive_batch(b64, jobs64, stream=st64)
        g64.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(8):
            g64.replay()
        e1.record()
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / 8
        b64.close()
        assert plan.device_status() == 0
        batch64 = {"subframes": n64, "ms_per_batch": ms64, "res_per_s": n64 * res_per_step / (ms64 * 1e-3),
                   "api": "rapro_receive_batch, 8 streams, one CUDA graph per batch"}
        del jobs64

    # comb pilots (Sec. II, IV-B) on the same 128 x 12 x 1200 shape: 12W, 3W, interpolated LS
    comb = {}
    if want("comb") and rank == 0 and world == 1:
        S = 12
        csets = []
        for i in range(N_SETS):
            sf = synth.make_comb_subframe(sh, seed=synth.SEED_BASE + 2000 + i, S=S)
            csets.append({k: torch.from_numpy(synth.as_c64(sf[k])).to(dev) for k in ("y_pilot", "pilots", "y_data")})
        for mname, method in (("12W", R.RAPRO_COMB_SW), ("3W", R.RAPRO_COMB_3W), ("interp3_ls", R.RAPRO_COMB_INTERP3)):
            pc = R.make_params(M=sh.M, K=sh.K, n_sc=sh.n_sc, n_fft=sh.n_fft, subblock=0, sigma2=sh.sigma2,
                               qam_bits=sh.qam_bits, n_taps=sh.n_taps, tau_rms=sh.tau_rms,
                               pilot_layout=R.RAPRO_PILOT_COMB, comb_spacing=S, comb_method=method)
            with R.Plan(pc) as plc:
                def cstep(i, det=True, stream=None):
                    d, o = csets[i % N_SETS], outs[i % IN_FLIGHT]
                    R.rapro_ce_comb(plc, d["y_pilot"], d["pilots"], o["h"], stream=stream)
                    if det:
                        R.rapro_mmse_detect(plc, o["h"], d["y_data"], o["x"], o["lab"], None, o["info"], stream=stream)

                def ccapture(det, pipelines):
                    g = torch.cuda.CUDAGraph()
                    st = torch.cuda.Stream()
                    side = [torch.cuda.Stream() for _ in range(pipelines)]
                    st.wait_stream(torch.cuda.current_stream())
                    with torch.cuda.stream(st):
                        with torch.cuda.graph(g, stream=st):
                            fork = torch.cuda.Event()
                            fork.record(st)
                            for q in side:
                                q.wait_event(fork)
                            for i in range(GRAPH_STEPS):
                                cstep(i, det, stream=side[i % pipelines])
                            for q in side:
                                join = torch.cuda.Event()
                                join.record(q)
                                st.wait_event(join)
                    torch.cuda.synchronize()
                    return g
                for i in range(3):
                    cstep(i)
                torch.cuda.synchronize()
                gc_full, gc_est = ccapture(True, IN_FLIGHT), ccapture(False, 1)
                us_full = time_graph(gc_full, 64)
                us_c = time_graph(gc_est, 64)
                cb = 8 * (sh.n_slots * sh.M * sh.n_sc + sh.n_slots * sh.n_sc + sh.n_slots * sh.K * sh.M * sh.n_sc)
                comb[mname] = {"res_per_s": res_per_step / (us_full * 1e-6), "estimator_us": us_c,
                               "estimator_alg_bytes": cb, "estimator_hbm_frac": cb / (us_c * 1e-6) / (peaks()[0] * 1e9)}
                assert plc.device_status() == 0

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    value = whole_job_value(world, res_per_step, args.steps, ms)
    hbm, peak_kind = peaks()
    rows = {}
    # the estimator runs on the tensor cores (3 TF32 passes) for every even B <= 2048 dividing
    # n_sc; its compute roof is then the tensor rate, not the FP32 FMA rate
    est_on_tc = B % 2 == 0 and sh.n_sc % B == 0 and B <= 2048
    tc_src = tf32x3_peak()[1]
    alu_peak = ffma["tflops"]
    for name, us in (("ls_lmmse", us_est), ("detect", us_det)):
        rows[name] = roof_row(alg[name], us, hbm, name == "ls_lmmse" and est_on_tc, alu_peak)
    dom = max(rows, key=lambda k: rows[k]["us_per_launch"])
    r = rows[dom]
    traffic = measured_traffic(dom)
    roof = {"bound": r["bound"], "achieved": r["achieved"], "peak": r["peak"], "unit": r["unit"],
            "frac": r["frac"], "traffic": traffic, "kernel": dom,
            "peak_source": (f"{peak_kind} HBM copy bandwidth" if r["bound"] == "hbm" else
                            tc_src if r["bound"] == "tensor" else
                            "measured FP32 FMA peak (rapro_measure_ffma_peak)")}
    # The path against its roofline.  Binding form: the estimator's flops run on the tensor
    # cores (3 TF32 passes) when est_on_tc, the detector's on FP32 FMA; the units work side
    # by side, so t_roof = max(bytes / HBM, estimator flops / its unit, detector flops / FMA).
    # The all-FMA form (every flop on FP32 FMA) is given beside it.
    pa = alg["path"]
    t_step = ms / args.steps * 1e-3
    tc_peak = tf32x3_peak()[0]
    t_bytes = pa["bytes"] / (hbm * 1e9)
    t_est = alg["ls_lmmse"]["flops"] / ((tc_peak if est_on_tc else alu_peak) * 1e12)
    t_det = alg["detect"]["flops"] / (alu_peak * 1e12)
    terms = {"hbm": t_bytes, "tensor" if est_on_tc else "alu_estimator": t_est, "alu_detector": t_det}
    bind = max(terms, key=terms.get)
    t_roof = terms[bind]
    t_fma = max(t_bytes, pa["flops"] / (alu_peak * 1e12))
    path_roof = {"bound": bind, "alg_bytes": pa["bytes"], "alg_flops": pa["flops"], "t_roof_us": t_roof * 1e6,
                 "t_step_us": t_step * 1e6, "frac": t_roof / t_step,
                 "terms_us": {k: v * 1e6 for k, v in terms.items()},
                 "all_fma_form": {"t_roof_us": t_fma * 1e6, "frac": t_fma / t_step,
                                  "bound": "hbm" if t_bytes >= t_fma else "alu"},
                 "note": "whole step (estimator + detector, subframes in flight) against max(algorithmic bytes / "
                         "HBM peak, estimator flops / the unit it runs on, detector flops / measured FP32 FMA "
                         "peak); all_fma_form puts every flop on FP32 FMA"}
    ev, dsplit, egrid = R.rapro_plan_variant(plan)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: seeded Rayleigh taps, exponential PDP, unit-modulus pilots, uniform 16-QAM payload, AWGN",
            "config": {"workload": desc, "M": sh.M, "K": sh.K, "n_sc": sh.n_sc, "subblock": B, "snr_db": sh.snr_db,
                       "res_per_step": res_per_step, "parallelism": f"replicas x{world}",
                       "l2": f"{N_SETS} resident input subframes rotated ({N_SETS * in_bytes / 2**20:.0f} MiB > "
                             f"{L2_BYTES / 2**20:.0f} MiB L2)",
                       "launch": f"graphs of exactly {args.steps} steps (pieces of <= {MAX_GRAPH_STEPS}); "
                                 f"consecutive steps rotate over {IN_FLIGHT} streams, so {IN_FLIGHT} "
                                 "subframes are in flight at any step count",
                       "plan_variant": {"est_variant": ev, "det_split": dsplit, "est_ctas_per_sm": egrid}},
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": whole_job_value(world, res_per_step, args.e2e_steps, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "Receiver.receive_host (pinned host in/out, rapro_receive_subframe; 2 buffer sets "
                           "so one subframe's copies overlap the previous one's kernels)",
                    "host_link_gbs": h2d * args.e2e_steps / (e2e_ms * 1e-3) / 1e9},
            "gpu_launches": 2 * args.steps, "clocks": clk, "ffma_peak": ffma,
            "path_roofline": path_roof,
            "kernels": rows, "kernel_timing": f"graphs of {GRAPH_STEPS} launches of one kernel alone on one "
                                              "stream, same plan variant as the timed step",
            "sweep_res_per_s": sweep, "user_symbols_per_s": value * sh.K,
            "comb_pilots": comb, "precision_form": prec, "differentiable": diff,
            "batched_heterogeneous": hetero, "batch_of_64_subframes": batch64}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_rapro(args)


if __name__ == "__main__":
    main()
