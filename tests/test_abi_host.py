"""CPU tests of the C-ABI library: it builds, loads, exports what rapro.h declares, and its
host-side logic (parameter checks, FP64 weights) behaves.  No GPU calls."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1802_05427_gb300 import _build, synth
from paper_1802_05427_gb300 import rapro as R
from oracle import rapro_oracle as O

from _common import params_for, oracle_r


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return R.lib()


def test_library_exports_every_declared_symbol(lib):
    names = R.header_functions()
    assert len(names) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", R.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_status_strings(lib):
    for code, name in ((0, "RAPRO_OK"), (1, "RAPRO_ERR_INVALID_ARG"), (3, "RAPRO_ERR_NOT_POSDEF"),
                       (4, "RAPRO_ERR_TIMEOUT")):
        assert lib.rapro_status_string(code).decode() == name


def _good():
    return params_for(synth.TINY, 12)


@pytest.mark.parametrize("field,value,expect", [
    ("M", 0, R.RAPRO_ERR_INVALID_ARG), ("K", 0, R.RAPRO_ERR_INVALID_ARG), ("K", 17, R.RAPRO_ERR_INVALID_ARG),
    ("n_sc", 0, R.RAPRO_ERR_INVALID_ARG), ("n_fft", 64, R.RAPRO_ERR_INVALID_ARG),
    ("subblock", 0, R.RAPRO_ERR_INVALID_ARG), ("subblock", 73, R.RAPRO_ERR_INVALID_ARG),
    ("sigma2", 0.0, R.RAPRO_ERR_INVALID_ARG), ("sigma2", -1.0, R.RAPRO_ERR_INVALID_ARG),
    ("sigma2", float("nan"), R.RAPRO_ERR_INVALID_ARG), ("qam_bits", 3, R.RAPRO_ERR_INVALID_ARG),
    ("n_taps", 0, R.RAPRO_ERR_INVALID_ARG), ("tau_rms", 0.0, R.RAPRO_ERR_INVALID_ARG),
    ("pdp", 7, R.RAPRO_ERR_INVALID_ARG), ("n_sym", 15, R.RAPRO_ERR_INVALID_ARG),
    ("n_sym", 30, R.RAPRO_ERR_INVALID_ARG), ("n_pilot_sym", 0, R.RAPRO_ERR_INVALID_ARG),
    ("pilot_layout", 7, R.RAPRO_ERR_INVALID_ARG),
])
def test_params_validation(lib, field, value, expect):
    p = _good()
    assert R.rapro_params_validate(p) == R.RAPRO_OK
    setattr(p, field, value)
    assert R.rapro_params_validate(p) == expect
    assert lib.rapro_last_error().decode()


def test_pilot_index_must_sit_inside_its_slot(lib):
    p = _good()
    p.pilot_sym_idx[1] = 3
    assert R.rapro_params_validate(p) == R.RAPRO_ERR_INVALID_ARG


@pytest.mark.parametrize("B", [1, 5, 12, 48, 100])
@pytest.mark.parametrize("pdp", ["exp", "uniform_L"])
def test_host_fp64_weights_match_oracle(lib, B, pdp):
    """The library's FP64 Cholesky-based W equals the oracle's LU-based W (Eq. 13/17)."""
    sh = synth.PAPER_SCALE
    p = params_for(sh, min(B, sh.n_sc), pdp=pdp)
    W = R.rapro_build_weights_host(p, B)
    idx = np.arange(B)
    Rb = O.corr_matrix(idx, idx, oracle_r(sh, pdp))
    Wo = O.lmmse_weight(Rb, Rb, sh.sigma2)
    np.testing.assert_allclose(W, Wo, rtol=0, atol=1e-10 * max(1.0, np.abs(Wo).max()))


def test_host_weights_reject_bad_block(lib):
    with pytest.raises(R.RaproError):
        R.rapro_build_weights_host(_good(), 0)


# ------------------------------------------------------------------ comb layout
def _comb(method=R.RAPRO_COMB_SW, S=12, sh=synth.PAPER_SCALE, pdp="exp"):
    p = params_for(sh, 1, pdp=pdp)
    p.pilot_layout, p.comb_spacing, p.comb_method = R.RAPRO_PILOT_COMB, S, method
    p.subblock = 0                                    # unused by comb plans
    return p


@pytest.mark.parametrize("field,value", [
    ("comb_spacing", 11), ("comb_spacing", 17), ("comb_spacing", 7), ("comb_method", 5), ("n_sc", 132),
])
def test_comb_params_validation(lib, field, value):
    """K <= S <= 16, S | n_sc, enough tones for the window, a known method."""
    p = _comb()
    assert R.rapro_params_validate(p) == R.RAPRO_OK
    setattr(p, field, value)
    assert R.rapro_params_validate(p) == R.RAPRO_ERR_INVALID_ARG
    assert lib.rapro_last_error().decode()


def test_comb_3w_needs_three_dividing_the_spacing(lib):
    p = _comb(R.RAPRO_COMB_3W, S=16)
    assert R.rapro_params_validate(p) == R.RAPRO_ERR_INVALID_ARG
    p = _comb(R.RAPRO_COMB_INTERP3, S=12)
    assert R.rapro_params_validate(p) == R.RAPRO_OK


@pytest.mark.parametrize("method", [R.RAPRO_COMB_3W, R.RAPRO_COMB_SW])
@pytest.mark.parametrize("pdp", ["exp", "uniform_L"])
def test_host_comb_weights_match_oracle(lib, method, pdp):
    """The library's FP64 comb weights (Cholesky) equal the oracle's per-group W (LU), for
    every weight index and user, mapped through the oracle's group tables."""
    sh = synth.PAPER_SCALE
    S, N = 12, sh.n_sc
    p = _comb(method, S, pdp=pdp)
    W = R.rapro_build_comb_weights_host(p)
    r = oracle_r(sh, pdp)
    om = O.COMB_SW if method == R.RAPRO_COMB_SW else O.COMB_3W
    Q = S if method == R.RAPRO_COMB_SW else 3
    for k in range(sh.K):
        tones = O.comb_tones(k, S, N)
        seen = set()
        for o, i0, widx in O.comb_groups(om, k, S, N):
            if widx in seen:
                continue
            seen.add(widx)
            Wo = O.comb_weight(o, tones[i0:i0 + Q], r, sh.sigma2)
            got = W[k if method == R.RAPRO_COMB_SW else 0, widx]
            np.testing.assert_allclose(got, Wo, rtol=0, atol=1e-10 * max(1.0, np.abs(Wo).max()))
        assert seen == set(range(Q))


# ------------------------------------------------------------- precision form
def test_precision_validation(lib):
    p = params_for(synth.PAPER_SCALE, 12)
    p.precision = R.RAPRO_PREC_BF16
    assert R.rapro_params_validate(p) == R.RAPRO_OK
    for B in (7, 13, 1199):                # odd, not dividing 1200
        p.subblock = B
        assert R.rapro_params_validate(p) == R.RAPRO_ERR_UNSUPPORTED
    for B in (48, 100, 1200):              # the large-block tensor-core GEMM
        p.subblock = B
        assert R.rapro_params_validate(p) == R.RAPRO_OK
    p.subblock, p.precision = 12, R.RAPRO_PREC_FP16
    assert R.rapro_params_validate(p) == R.RAPRO_OK
    for B in (7, 13, 1199):
        p.subblock = B
        assert R.rapro_params_validate(p) == R.RAPRO_ERR_UNSUPPORTED
    p.subblock, p.precision = 12, 5
    assert R.rapro_params_validate(p) == R.RAPRO_ERR_INVALID_ARG


# --------------------------------------------------------- weight gradient (host)
@pytest.mark.parametrize("B", [1, 5, 12, 30])
def test_host_weight_gradient_matches_autograd(lib, B):
    """rapro_weight_grad_host: 2 Re sum conj(G) dW/dtheta equals torch.autograd of the same
    contraction through the differentiable oracle's W(sigma2, tau)."""
    import torch
    from oracle import rapro_grad_oracle as G
    sh = synth.SubframeShape(M=4, K=2, n_sc=62, n_fft=128, n_taps=7, tau_rms=2.5, snr_db=9.0)
    p = params_for(sh, B)
    rng = np.random.default_rng(B)
    tail = sh.n_sc % B
    gm = rng.standard_normal((B, B)) + 1j * rng.standard_normal((B, B))
    gt = rng.standard_normal((tail, tail)) + 1j * rng.standard_normal((tail, tail)) if tail else None
    d_s2, d_tau = R.rapro_weight_grad_host(p, gm, gt)
    s2 = torch.tensor(sh.sigma2, dtype=torch.float64, requires_grad=True)
    tau = torch.tensor(sh.tau_rms, dtype=torch.float64, requires_grad=True)
    f = 2 * torch.real(torch.sum(torch.conj(torch.as_tensor(gm)) * G.block_weight(B, s2, tau, sh.n_taps, sh.n_fft)))
    if tail:
        f = f + 2 * torch.real(torch.sum(torch.conj(torch.as_tensor(gt)) *
                                         G.block_weight(tail, s2, tau, sh.n_taps, sh.n_fft)))
    f.backward()
    np.testing.assert_allclose([d_s2, d_tau], [float(s2.grad), float(tau.grad)], rtol=1e-9, atol=1e-12)


NULL_HANDLE_CALLS = [
    ("rapro_plan_dims", 5), ("rapro_plan_device_status", 3), ("rapro_ce_ls", 5),
    ("rapro_ce_lmmse_subblock", 5), ("rapro_ce_ls_lmmse", 6), ("rapro_mmse_detect", 8),
    ("rapro_ce_comb", 5), ("rapro_receive_subframe", 10), ("rapro_mse_backward", 12),
    ("rapro_plan_tune", 7), ("rapro_plan_variant", 4), ("rapro_plan_set_variant", 4),
    ("rapro_plan_set_receive_form", 2), ("rapro_receive_is_fused", 4), ("rapro_receive_batch", 4),
    ("rapro_receive_subframe_noalloc", 9), ("rapro_plan_create", 2), ("rapro_batch_create", 2),
]


@pytest.mark.parametrize("name,n_args", NULL_HANDLE_CALLS, ids=[c[0] for c in NULL_HANDLE_CALLS])
def test_null_handles_are_rejected_before_any_device_work(lib, name, n_args):
    """A NULL plan, batch, params or output handle returns RAPRO_ERR_INVALID_ARG with a message;
    the check precedes every CUDA call, so it runs here without a GPU."""
    f = getattr(lib, name)
    assert len(f.argtypes) == n_args
    args = [0 if t is ctypes.c_int else None for t in f.argtypes]
    if name == "rapro_batch_create":
        args[0] = 1                                  # a valid stream count, NULL out
    assert f(*args) == R.RAPRO_ERR_INVALID_ARG
    assert lib.rapro_last_error().decode()


def test_null_destroy_is_a_no_op(lib):
    assert lib.rapro_plan_destroy(None) == R.RAPRO_OK
    assert lib.rapro_batch_destroy(None) == R.RAPRO_OK


def test_binding_fails_loudly_without_the_library(monkeypatch):
    """No CPU fallback: a missing librapro.so is an ImportError, not a silent path."""
    monkeypatch.setattr(R, "_lib", None)
    monkeypatch.setattr(R, "LIB_PATH", os.path.join(os.path.dirname(R.LIB_PATH), "no_such_librapro.so"))
    with pytest.raises(ImportError, match="missing"):
        R.lib()


def test_binding_rejects_host_tensors(lib):
    """Arrays must be CUDA tensors of the declared dtype, shape and layout; a host tensor is a
    TypeError raised before any library call (the kernels are the only compute path)."""
    import torch
    p = _good()
    T, D = p.n_pilot_sym, p.n_sym // p.n_pilot_sym - 1
    K, M, N = p.K, p.M, p.n_sc
    c64 = torch.complex64
    host = dict(y_pilot=torch.zeros(T, K, M, N, dtype=c64), pilots=torch.ones(T, K, N, dtype=c64),
                y_data=torch.zeros(T * D, M, N, dtype=c64), x_eq=torch.zeros(T * D, K, N, dtype=c64))
    with pytest.raises(TypeError, match="CUDA tensor"):
        R.rapro_receive_subframe_noalloc(p, **host)
    with pytest.raises(TypeError, match="CUDA tensor"):
        R._ptr(host["x_eq"], (T * D, K, N), c64, "x_eq")
    with pytest.raises(TypeError, match="CUDA tensor"):
        R._ptr(np.zeros((T * D, K, N), np.complex64), (T * D, K, N), c64, "x_eq")
