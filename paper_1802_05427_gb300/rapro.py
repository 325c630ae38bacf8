"""Python binding of librapro.so: the C-ABI entry points under the same names.

Argument marshalling only -- every step of the receive path runs in the CUDA library.
Tensors are torch tensors on the plan's CUDA device (complex64 for rapro_c32 arrays,
uint8 labels, float32 LLRs, int32 info), C-contiguous, in the layouts of rapro.h.
Streams default to torch's current stream.  The library must have been built
(``paper_1802_05427_gb300._build.build()``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Sequence

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librapro.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "rapro.h")

RAPRO_OK, RAPRO_ERR_INVALID_ARG, RAPRO_ERR_CUDA, RAPRO_ERR_NOT_POSDEF = 0, 1, 2, 3
RAPRO_ERR_TIMEOUT, RAPRO_ERR_UNSUPPORTED, RAPRO_ERR_NOMEM = 4, 5, 6
RAPRO_PILOT_ORTHOGONAL, RAPRO_PILOT_COMB = 0, 1
RAPRO_PDP_EXP, RAPRO_PDP_UNIFORM_L = 0, 1
RAPRO_COMB_3W, RAPRO_COMB_SW, RAPRO_COMB_INTERP3 = 0, 1, 2
RAPRO_PREC_FP32, RAPRO_PREC_BF16, RAPRO_PREC_FP16 = 0, 1, 2
RAPRO_RECV_SPLIT, RAPRO_RECV_FUSED = 0, 1
RAPRO_DET_REFINED, RAPRO_DET_FP32 = 0, 1
RAPRO_MAX_PILOT_SYM = 8


class RaproParams(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_int), ("K", ctypes.c_int), ("n_sc", ctypes.c_int), ("n_fft", ctypes.c_int),
        ("n_sym", ctypes.c_int), ("n_pilot_sym", ctypes.c_int),
        ("pilot_sym_idx", ctypes.c_int * RAPRO_MAX_PILOT_SYM),
        ("pilot_layout", ctypes.c_int), ("subblock", ctypes.c_int), ("sigma2", ctypes.c_double),
        ("pdp", ctypes.c_int), ("n_taps", ctypes.c_int), ("tau_rms", ctypes.c_double),
        ("L", ctypes.c_double), ("qam_bits", ctypes.c_int),
        ("comb_spacing", ctypes.c_int), ("comb_method", ctypes.c_int), ("precision", ctypes.c_int),
    ]


class RaproJob(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("y_pilot", ctypes.c_void_p), ("pilots", ctypes.c_void_p),
                ("y_data", ctypes.c_void_p), ("h_out", ctypes.c_void_p), ("x_eq", ctypes.c_void_p),
                ("labels", ctypes.c_void_p), ("llr", ctypes.c_void_p), ("info", ctypes.c_void_p)]


class RaproError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str):
        super().__init__(f"{what}: status {status}: {msg}")
        self.status = status


_lib = None
_P = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Load librapro.so (once) and declare the entry points' signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1802_05427_gb300._build.build()")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "rapro_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "rapro_last_error": ([], ctypes.c_char_p),
        "rapro_params_validate": ([ctypes.POINTER(RaproParams)], ctypes.c_int),
        "rapro_build_weights_host": ([ctypes.POINTER(RaproParams), ctypes.c_int, _P], ctypes.c_int),
        "rapro_build_comb_weights_host": ([ctypes.POINTER(RaproParams), _P], ctypes.c_int),
        "rapro_ce_comb": ([_P, _P, _P, _P, _P], ctypes.c_int),
        "rapro_mse_backward": ([_P] * 12, ctypes.c_int),
        "rapro_plan_tune": ([_P] * 7, ctypes.c_int),
        "rapro_plan_variant": ([_P, _P, _P, _P], ctypes.c_int),
        "rapro_plan_set_receive_form": ([_P, ctypes.c_int], ctypes.c_int),
        "rapro_plan_set_variant": ([_P, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "rapro_receive_is_fused": ([_P, _P, _P, _P], ctypes.c_int),
        "rapro_batch_create": ([ctypes.c_int, ctypes.POINTER(_P)], ctypes.c_int),
        "rapro_batch_destroy": ([_P], ctypes.c_int),
        "rapro_receive_batch": ([_P, ctypes.POINTER(RaproJob), ctypes.c_int, _P], ctypes.c_int),
        "rapro_weight_grad_host": ([ctypes.POINTER(RaproParams), _P, _P, _P], ctypes.c_int),
        "rapro_plan_create": ([ctypes.POINTER(RaproParams), ctypes.POINTER(_P)], ctypes.c_int),
        "rapro_plan_destroy": ([_P], ctypes.c_int),
        "rapro_plan_dims": ([_P, _P, _P, _P, _P], ctypes.c_int),
        "rapro_plan_device_status": ([_P, ctypes.c_int, _P], ctypes.c_int),
        "rapro_ce_ls": ([_P, _P, _P, _P, _P], ctypes.c_int),
        "rapro_ce_lmmse_subblock": ([_P, _P, _P, _P, _P], ctypes.c_int),
        "rapro_ce_ls_lmmse": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
        "rapro_mmse_detect": ([_P, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
        "rapro_receive_subframe": ([_P, _P, _P, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
        "rapro_receive_subframe_noalloc": ([ctypes.POINTER(RaproParams), _P, _P, _P, _P, _P, _P, _P, _P],
                                           ctypes.c_int),
        "rapro_noalloc_status": ([ctypes.c_int, _P, _P], ctypes.c_int),
        "rapro_gram_tc": ([_P, _P, _P, _P, ctypes.c_int, _P], ctypes.c_int),
        "rapro_plan_set_wait_test": ([_P, ctypes.c_int, ctypes.c_uint32], ctypes.c_int),
        "rapro_plan_set_detector_form": ([_P, ctypes.c_int], ctypes.c_int),
        "rapro_measure_ffma_peak": ([ctypes.c_int, _P, _P, _P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def header_functions(path: str = HEADER) -> list:
    """Names of the functions include/rapro.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rapro_[a-z_0-9]+)\s*\(", text)))


def _check(status: int, what: str) -> None:
    if status != RAPRO_OK:
        raise RaproError(status, what, lib().rapro_last_error().decode())


def make_params(*, M: int, K: int, n_sc: int, n_fft: int, subblock: int, sigma2: float,
                qam_bits: int, n_sym: int = 14, n_pilot_sym: int = 2,
                pilot_sym_idx: Optional[Sequence[int]] = None, pdp: int = RAPRO_PDP_EXP,
                n_taps: int = 6, tau_rms: float = 4.0, L: float = 8.0,
                pilot_layout: int = RAPRO_PILOT_ORTHOGONAL, comb_spacing: int = 0,
                comb_method: int = RAPRO_COMB_SW, precision: int = RAPRO_PREC_FP32) -> RaproParams:
    """Build a rapro_params; by default each slot's pilot sits in its 4th symbol (3, 10)."""
    p = RaproParams()
    p.M, p.K, p.n_sc, p.n_fft = M, K, n_sc, n_fft
    p.n_sym, p.n_pilot_sym = n_sym, n_pilot_sym
    slot = n_sym // n_pilot_sym if n_pilot_sym else 1
    idx = list(pilot_sym_idx) if pilot_sym_idx is not None else [j * slot + min(3, slot - 1)
                                                                  for j in range(n_pilot_sym)]
    for j, v in enumerate(idx[:RAPRO_MAX_PILOT_SYM]):
        p.pilot_sym_idx[j] = v
    p.pilot_layout, p.subblock, p.sigma2 = pilot_layout, subblock, sigma2
    p.pdp, p.n_taps, p.tau_rms, p.L, p.qam_bits = pdp, n_taps, tau_rms, L, qam_bits
    p.comb_spacing, p.comb_method, p.precision = comb_spacing, comb_method, precision
    return p


def rapro_params_validate(p: RaproParams) -> int:
    return lib().rapro_params_validate(ctypes.byref(p))


def rapro_build_weights_host(p: RaproParams, block_len: int):
    """FP64 W of one block (numpy complex128 [block_len][block_len])."""
    import numpy as np
    buf = np.zeros(2 * block_len * block_len, dtype=np.float64)
    _check(lib().rapro_build_weights_host(ctypes.byref(p), block_len, buf.ctypes.data),
           "rapro_build_weights_host")
    return (buf[0::2] + 1j * buf[1::2]).reshape(block_len, block_len)


def rapro_build_comb_weights_host(p: RaproParams):
    """FP64 comb weights (numpy complex128 [sets][Q][Q][Q]: set, weight index, row, column)."""
    import numpy as np
    Q = p.comb_spacing if p.comb_method == RAPRO_COMB_SW else 3
    sets = p.K if p.comb_method == RAPRO_COMB_SW else 1
    buf = np.zeros(2 * sets * Q ** 3, dtype=np.float64)
    _check(lib().rapro_build_comb_weights_host(ctypes.byref(p), buf.ctypes.data), "rapro_build_comb_weights_host")
    return (buf[0::2] + 1j * buf[1::2]).reshape(sets, Q, Q, Q)


class Plan:
    """Owns a rapro_plan (weights on the device, workspace, status word)."""

    def __init__(self, params: RaproParams):
        self.params = params
        h = _P()
        _check(lib().rapro_plan_create(ctypes.byref(params), ctypes.byref(h)), "rapro_plan_create")
        self.handle = h
        T, D, nb, tail = (ctypes.c_int() for _ in range(4))
        _check(lib().rapro_plan_dims(h, ctypes.byref(T), ctypes.byref(D), ctypes.byref(nb),
                                     ctypes.byref(tail)), "rapro_plan_dims")
        self.T, self.D, self.nb, self.tail = T.value, D.value, nb.value, tail.value

    def close(self) -> None:
        if getattr(self, "handle", None):
            _check(lib().rapro_plan_destroy(self.handle), "rapro_plan_destroy")
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_status(self, reset: bool = False) -> int:
        v = ctypes.c_int()
        _check(lib().rapro_plan_device_status(self.handle, int(reset), ctypes.byref(v)),
               "rapro_plan_device_status")
        return v.value

    # shapes of the C-ABI arrays
    def shapes(self) -> dict:
        p = self.params
        T, D, K, M, N, q = self.T, self.D, p.K, p.M, p.n_sc, p.qam_bits
        comb = p.pilot_layout == RAPRO_PILOT_COMB
        return dict(y_pilot=(T, M, N) if comb else (T, K, M, N), pilots=(T, N) if comb else (T, K, N),
                    y_data=(T * D, M, N), h=(T, K, M, N),
                    x_eq=(T * D, K, N), labels=(T * D, K, N), llr=(T * D, K, N, q), info=(T, N))


def _ptr(t, shape, dtype, name):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def rapro_ce_ls(plan: Plan, y_pilot, pilots, h_ls, stream=None) -> None:
    import torch
    s = plan.shapes()
    c64 = torch.complex64
    _check(lib().rapro_ce_ls(plan.handle, _ptr(y_pilot, s["y_pilot"], c64, "y_pilot"),
                             _ptr(pilots, s["pilots"], c64, "pilots"), _ptr(h_ls, s["h"], c64, "h_ls"),
                             _stream(stream)), "rapro_ce_ls")


def rapro_ce_lmmse_subblock(plan: Plan, h_ls, h, w_override=None, stream=None) -> None:
    import torch
    s = plan.shapes()
    c64 = torch.complex64
    _check(lib().rapro_ce_lmmse_subblock(plan.handle, _ptr(h_ls, s["h"], c64, "h_ls"),
                                         _w_override(plan, w_override),
                                         _ptr(h, s["h"], c64, "h"), _stream(stream)),
           "rapro_ce_lmmse_subblock")


def _w_override(plan: Plan, w_override):
    import torch
    if w_override is None:
        return None
    B, tail, nb = plan.params.subblock, plan.tail, plan.nb
    n_w = (nb - (1 if tail else 0)) * B * B + tail * tail
    return _ptr(w_override, (n_w,), torch.complex64, "w_override")


def rapro_ce_ls_lmmse(plan: Plan, y_pilot, pilots, h, w_override=None, stream=None) -> None:
    import torch
    s = plan.shapes()
    c64 = torch.complex64
    _check(lib().rapro_ce_ls_lmmse(plan.handle, _ptr(y_pilot, s["y_pilot"], c64, "y_pilot"),
                                   _ptr(pilots, s["pilots"], c64, "pilots"), _w_override(plan, w_override),
                                   _ptr(h, s["h"], c64, "h"), _stream(stream)), "rapro_ce_ls_lmmse")


def rapro_ce_comb(plan: Plan, y_pilot, pilots, h, stream=None) -> None:
    import torch
    s = plan.shapes()
    c64 = torch.complex64
    _check(lib().rapro_ce_comb(plan.handle, _ptr(y_pilot, s["y_pilot"], c64, "y_pilot"),
                               _ptr(pilots, s["pilots"], c64, "pilots"), _ptr(h, s["h"], c64, "h"),
                               _stream(stream)), "rapro_ce_comb")


def rapro_mse_backward(plan: Plan, y_pilot, pilots, y_data, h, x_eq, x_ref, g_h, scalars, g_w_main,
                       g_w_tail=None, stream=None) -> None:
    import torch
    s = plan.shapes()
    c64 = torch.complex64
    B, tail = plan.params.subblock, plan.tail
    _check(lib().rapro_mse_backward(plan.handle, _ptr(y_pilot, s["y_pilot"], c64, "y_pilot"),
                                    _ptr(pilots, s["pilots"], c64, "pilots"), _ptr(y_data, s["y_data"], c64, "y_data"),
                                    _ptr(h, s["h"], c64, "h"), _ptr(x_eq, s["x_eq"], c64, "x_eq"),
                                    _ptr(x_ref, s["x_eq"], c64, "x_ref"), _ptr(g_h, s["h"], c64, "g_h"),
                                    _ptr(scalars, (2,), torch.float32, "scalars"),
                                    _ptr(g_w_main, (B, B), c64, "g_w_main"),
                                    _ptr(g_w_tail, (tail, tail), c64, "g_w_tail") if tail else None,
                                    _stream(stream)), "rapro_mse_backward")


def rapro_plan_tune(plan: Plan, y_pilot, pilots, y_data, h, x_eq, stream=None) -> None:
    import torch
    s = plan.shapes()
    c64 = torch.complex64
    _check(lib().rapro_plan_tune(plan.handle, _ptr(y_pilot, s["y_pilot"], c64, "y_pilot"),
                                 _ptr(pilots, s["pilots"], c64, "pilots"), _ptr(y_data, s["y_data"], c64, "y_data"),
                                 _ptr(h, s["h"], c64, "h"), _ptr(x_eq, s["x_eq"], c64, "x_eq"), _stream(stream)),
           "rapro_plan_tune")


def rapro_plan_variant(plan: Plan):
    """(estimator kernel, detector warps per role, tensor-core estimator CTAs per SM)."""
    ev, ds, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().rapro_plan_variant(plan.handle, ctypes.byref(ev), ctypes.byref(ds), ctypes.byref(g)),
           "rapro_plan_variant")
    return ev.value, ds.value, g.value


def rapro_plan_set_variant(plan: Plan, est_variant: int, det_split: int, est_ctas_per_sm: int = 1) -> None:
    _check(lib().rapro_plan_set_variant(plan.handle, int(est_variant), int(det_split), int(est_ctas_per_sm)),
           "rapro_plan_set_variant")


def rapro_plan_set_receive_form(plan: Plan, form: int) -> None:
    _check(lib().rapro_plan_set_receive_form(plan.handle, int(form)), "rapro_plan_set_receive_form")


def rapro_receive_is_fused(plan: Plan, y_pilot, y_data) -> bool:
    """Whether rapro_receive_subframe with these tensors runs the fused kernel."""
    import torch
    s = plan.shapes()
    c64 = torch.complex64
    f = ctypes.c_int()
    _check(lib().rapro_receive_is_fused(plan.handle, _ptr(y_pilot, s["y_pilot"], c64, "y_pilot"),
                                        _ptr(y_data, s["y_data"], c64, "y_data"), ctypes.byref(f)),
           "rapro_receive_is_fused")
    return bool(f.value)


class Batch:
    """A pool of CUDA streams for rapro_receive_batch."""

    def __init__(self, n_streams: int = 8):
        h = _P()
        _check(lib().rapro_batch_create(int(n_streams), ctypes.byref(h)), "rapro_batch_create")
        self.handle = h

    def close(self) -> None:
        if getattr(self, "handle", None):
            _check(lib().rapro_batch_destroy(self.handle), "rapro_batch_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rapro_receive_batch(batch: Batch, jobs: list, stream=None) -> None:
    """jobs: dicts with plan (Plan) and the tensors of rapro_receive_subframe
    (y_pilot, pilots, y_data, x_eq; optional h_out, labels, llr, info)."""
    import torch
    arr = (RaproJob * len(jobs))()
    c64 = torch.complex64
    for i, j in enumerate(jobs):
        pl = j["plan"]
        s = pl.shapes()
        arr[i].plan = pl.handle.value
        arr[i].y_pilot = _ptr(j["y_pilot"], s["y_pilot"], c64, "y_pilot").value
        arr[i].pilots = _ptr(j["pilots"], s["pilots"], c64, "pilots").value
        arr[i].y_data = _ptr(j["y_data"], s["y_data"], c64, "y_data").value
        arr[i].x_eq = _ptr(j["x_eq"], s["x_eq"], c64, "x_eq").value
        for name, shape, dt in (("h_out", s["h"], c64), ("labels", s["labels"], torch.uint8),
                                ("llr", s["llr"], torch.float32), ("info", s["info"], torch.int32)):
            v = _ptr(j.get(name), shape, dt, name)
            setattr(arr[i], name, None if v is None else v.value)
    _check(lib().rapro_receive_batch(batch.handle, arr, len(jobs), _stream(stream)), "rapro_receive_batch")


def rapro_weight_grad_host(p: RaproParams, g_w_main, g_w_tail=None):
    """(dL/dsigma2, dL/dtau_rms) through the estimator weights, FP64 on the host."""
    import numpy as np
    gm = np.ascontiguousarray(np.asarray(g_w_main, dtype=np.complex128)).view(np.float64)
    gt = None if g_w_tail is None else np.ascontiguousarray(np.asarray(g_w_tail, dtype=np.complex128)).view(np.float64)
    out = np.zeros(2, dtype=np.float64)
    _check(lib().rapro_weight_grad_host(ctypes.byref(p), gm.ctypes.data, None if gt is None else gt.ctypes.data,
                                        out.ctypes.data), "rapro_weight_grad_host")
    return float(out[0]), float(out[1])


def rapro_mmse_detect(plan: Plan, h, y_data, x_eq, labels=None, llr=None, info=None, stream=None) -> None:
    import torch
    s = plan.shapes()
    c64 = torch.complex64
    _check(lib().rapro_mmse_detect(plan.handle, _ptr(h, s["h"], c64, "h"),
                                   _ptr(y_data, s["y_data"], c64, "y_data"),
                                   _ptr(x_eq, s["x_eq"], c64, "x_eq"),
                                   _ptr(labels, s["labels"], torch.uint8, "labels"),
                                   _ptr(llr, s["llr"], torch.float32, "llr"),
                                   _ptr(info, s["info"], torch.int32, "info"), _stream(stream)),
           "rapro_mmse_detect")


def rapro_receive_subframe(plan: Plan, y_pilot, pilots, y_data, x_eq, labels=None, llr=None,
                           info=None, h_out=None, stream=None) -> None:
    import torch
    s = plan.shapes()
    c64 = torch.complex64
    _check(lib().rapro_receive_subframe(plan.handle, _ptr(y_pilot, s["y_pilot"], c64, "y_pilot"),
                                        _ptr(pilots, s["pilots"], c64, "pilots"),
                                        _ptr(y_data, s["y_data"], c64, "y_data"),
                                        _ptr(h_out, s["h"], c64, "h_out"),
                                        _ptr(x_eq, s["x_eq"], c64, "x_eq"),
                                        _ptr(labels, s["labels"], torch.uint8, "labels"),
                                        _ptr(llr, s["llr"], torch.float32, "llr"),
                                        _ptr(info, s["info"], torch.int32, "info"), _stream(stream)),
           "rapro_receive_subframe")


def rapro_receive_subframe_noalloc(params: RaproParams, y_pilot, pilots, y_data, x_eq, labels=None,
                                   llr=None, info=None, stream=None) -> None:
    """The allocation-free receive: no plan, the library's fixed device scratch (see rapro.h)."""
    import torch
    p = params
    T, D = p.n_pilot_sym, p.n_sym // p.n_pilot_sym - 1
    K, M, N, q = p.K, p.M, p.n_sc, p.qam_bits
    c64 = torch.complex64
    _check(lib().rapro_receive_subframe_noalloc(
        ctypes.byref(p), _ptr(y_pilot, (T, K, M, N), c64, "y_pilot"), _ptr(pilots, (T, K, N), c64, "pilots"),
        _ptr(y_data, (T * D, M, N), c64, "y_data"), _ptr(x_eq, (T * D, K, N), c64, "x_eq"),
        _ptr(labels, (T * D, K, N), torch.uint8, "labels"), _ptr(llr, (T * D, K, N, q), torch.float32, "llr"),
        _ptr(info, (T, N), torch.int32, "info"), _stream(stream)), "rapro_receive_subframe_noalloc")


def rapro_plan_set_detector_form(plan: Plan, form: int) -> None:
    _check(lib().rapro_plan_set_detector_form(plan.handle, int(form)), "rapro_plan_set_detector_form")


def rapro_plan_set_wait_test(plan: Plan, stall_producer: bool, wait_rounds: int) -> None:
    """Diagnostics of the timeout path: short producer/consumer waits and a silent producer."""
    _check(lib().rapro_plan_set_wait_test(plan.handle, int(bool(stall_producer)), int(wait_rounds)),
           "rapro_plan_set_wait_test")


def rapro_gram_tc(plan: Plan, h, y_data, gram, fp16: bool = False, stream=None) -> None:
    """Gram and matched filter on the tensor cores (16-bit operands): gram [T][n_sc][K][K + D]."""
    import torch
    s = plan.shapes()
    c64 = torch.complex64
    T, K, N, D = plan.T, plan.params.K, plan.params.n_sc, plan.D
    _check(lib().rapro_gram_tc(plan.handle, _ptr(h, s["h"], c64, "h"), _ptr(y_data, s["y_data"], c64, "y_data"),
                               _ptr(gram, (T, N, K, K + D), c64, "gram"), int(bool(fp16)), _stream(stream)),
           "rapro_gram_tc")


def rapro_noalloc_status(reset: bool = False, stream=None) -> int:
    """Status word of the allocation-free receive on the current device (0 or RAPRO_ERR_TIMEOUT)."""
    v = ctypes.c_int(-1)
    _check(lib().rapro_noalloc_status(int(reset), ctypes.byref(v), _stream(stream)), "rapro_noalloc_status")
    return v.value


def rapro_measure_ffma_peak(trips: int = 50000, stream=None) -> tuple:
    """(TFLOP/s, ms) of the library's FP32 FMA-chain probe on the current device."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().rapro_measure_ffma_peak(int(trips), ctypes.byref(tf), ctypes.byref(ms), _stream(stream)),
           "rapro_measure_ffma_peak")
    return tf.value, ms.value


class Receiver:
    """A plan plus device buffers for subframes arriving in host memory: the call a user makes.

    ``receive_host`` copies pinned host inputs to the device, runs rapro_receive_subframe and
    copies the equalised symbols and labels back, all enqueued without waiting.  ``depth``
    buffer sets on their own streams are used in turn, so the copies of one subframe overlap
    the kernels of the previous one (the host link, not the kernels, bounds this path).
    ``join`` makes a stream (default: the current one) wait for everything enqueued so far;
    host output buffers of subframes still in flight must not be reused before that.
    """

    def __init__(self, params: RaproParams, device: int = 0, want_llr: bool = False, depth: int = 2):
        import torch
        torch.cuda.set_device(device)
        self.plan = Plan(params)
        s = self.plan.shapes()
        dev = torch.device("cuda", device)
        self.dev = dev
        self.slots = []
        for _ in range(max(1, depth)):
            self.slots.append(dict(
                y_pilot=torch.empty(s["y_pilot"], dtype=torch.complex64, device=dev),
                pilots=torch.empty(s["pilots"], dtype=torch.complex64, device=dev),
                y_data=torch.empty(s["y_data"], dtype=torch.complex64, device=dev),
                h=torch.empty(s["h"], dtype=torch.complex64, device=dev),
                x_eq=torch.empty(s["x_eq"], dtype=torch.complex64, device=dev),
                labels=torch.empty(s["labels"], dtype=torch.uint8, device=dev),
                llr=torch.empty(s["llr"], dtype=torch.float32, device=dev) if want_llr else None,
                info=torch.empty(s["info"], dtype=torch.int32, device=dev),
                stream=torch.cuda.Stream(device=dev)))
        self._next = 0
        first = self.slots[0]
        # single-slot views kept for callers that fill the device buffers themselves
        self.y_pilot, self.pilots, self.y_data = first["y_pilot"], first["pilots"], first["y_data"]
        self.x_eq, self.labels, self.llr, self.info = first["x_eq"], first["labels"], first["llr"], first["info"]

    def run_device(self, stream=None, slot=None) -> None:
        sl = self.slots[0] if slot is None else slot
        rapro_receive_subframe(self.plan, sl["y_pilot"], sl["pilots"], sl["y_data"], sl["x_eq"], sl["labels"],
                               sl["llr"], sl["info"], h_out=sl["h"], stream=stream)

    def fork(self, stream=None) -> None:
        """Every slot stream waits for ``stream`` (default: the current stream)."""
        import torch
        src = torch.cuda.current_stream(self.dev) if stream is None else stream
        for sl in self.slots:
            sl["stream"].wait_stream(src)

    def join(self, stream=None) -> None:
        """``stream`` (default: the current stream) waits for every slot stream."""
        import torch
        dst = torch.cuda.current_stream(self.dev) if stream is None else stream
        for sl in self.slots:
            dst.wait_stream(sl["stream"])

    def receive_host(self, y_pilot_h, pilots_h, y_data_h, x_eq_h, labels_h) -> None:
        import torch
        sl = self.slots[self._next]
        self._next = (self._next + 1) % len(self.slots)
        st = sl["stream"]
        with torch.cuda.stream(st):
            sl["y_pilot"].copy_(y_pilot_h, non_blocking=True)
            sl["pilots"].copy_(pilots_h, non_blocking=True)
            sl["y_data"].copy_(y_data_h, non_blocking=True)
            self.run_device(st, sl)
            x_eq_h.copy_(sl["x_eq"], non_blocking=True)
            labels_h.copy_(sl["labels"], non_blocking=True)
