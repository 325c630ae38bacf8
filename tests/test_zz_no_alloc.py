"""The allocation-free receive entry point against the plan-based one and the oracle (GPU).

rapro_receive_subframe_noalloc serves callers that cannot allocate device memory when a
subframe arrives: real-time slot loops that must not wait on an allocator, processes whose
device memory belongs to another framework's pool, and deployments that forbid run-time
allocation.  It uses the library's fixed device scratch instead of a plan's workspace.  It
must give the same results as rapro_receive_subframe with h_out == NULL, call after call,
match the FP64 oracle like the plan path does, report its status word, and refuse what does
not fit its scratch.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rapro_oracle as O
from paper_1802_05427_gb300 import _build, synth
from paper_1802_05427_gb300 import rapro as R

from _common import assert_parity, oracle_r, params_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()
    R.lib()
    torch.cuda.set_device(0)


def _run(fn, sf, sh):
    dev = torch.device("cuda", 0)
    ins = [torch.from_numpy(synth.as_c64(sf[k])).to(dev) for k in ("y_pilot", "pilots", "y_data")]
    T, D = sh.n_slots, sh.n_data_per_slot
    x = torch.full((T * D, sh.K, sh.n_sc), float("nan"), dtype=torch.complex64, device=dev)
    lab = torch.zeros((T * D, sh.K, sh.n_sc), dtype=torch.uint8, device=dev)
    llr = torch.zeros((T * D, sh.K, sh.n_sc, sh.qam_bits), dtype=torch.float32, device=dev)
    info = torch.full((T, sh.n_sc), -1, dtype=torch.int32, device=dev)
    fn(*ins, x, lab, llr, info)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in (x, lab, llr, info)]


@pytest.mark.parametrize("sh,B", [(synth.PAPER_SCALE, 12),
                                  (synth.SubframeShape(M=20, K=5, n_sc=100, n_fft=256, qam_bits=6), 7)])
def test_noalloc_matches_plan_receive_on_consecutive_calls(sh, B):
    params = params_for(sh, B)
    plan = R.Plan(params)
    for seed in (synth.SEED_BASE + 21, synth.SEED_BASE + 22):      # two calls in a row
        sf = synth.make_subframe(sh, seed=seed)
        ref = _run(lambda yp, p, yd, x, lab, llr, info: R.rapro_receive_subframe(plan, yp, p, yd, x, lab, llr, info),
                   sf, sh)
        got = _run(lambda yp, p, yd, x, lab, llr, info:
                   R.rapro_receive_subframe_noalloc(params, yp, p, yd, x, lab, llr, info), sf, sh)
        assert_parity(got[0], ref[0], (2,), 1e-5, what="x_eq vs plan path")
        np.testing.assert_array_equal(got[1], ref[1])
        np.testing.assert_allclose(got[2], ref[2], rtol=1e-4, atol=1e-3)
        np.testing.assert_array_equal(got[3], np.zeros_like(got[3]))
        assert R.rapro_noalloc_status(reset=True) == R.RAPRO_OK
        # and against the FP64 oracle on the same complex64 inputs
        c = {k: synth.as_c64(sf[k]).astype(np.complex128) for k in ("y_pilot", "pilots", "y_data")}
        o = O.receive_subframe(c["y_pilot"], c["pilots"], c["y_data"], B=B, sigma2=sh.sigma2, r=oracle_r(sh),
                               n_data_per_slot=sh.n_data_per_slot, q=sh.qam_bits)
        assert_parity(got[0], o["x_eq"], (2,), 1e-5, what="x_eq vs oracle")
        safe = O.boundary_margin(o["xhat"], sh.qam_bits) > 1e-4
        np.testing.assert_array_equal(got[1][safe], o["labels"][safe])
    plan.close()


def test_noalloc_rejects_what_does_not_fit():
    lib = R.lib()
    big = params_for(synth.SubframeShape(M=256, K=16, n_sc=1200, n_fft=2048, qam_bits=4), 12)
    assert lib.rapro_receive_subframe_noalloc(ctypes.byref(big), 8, 8, 8, 8, None, None, None, None) == \
        R.RAPRO_ERR_INVALID_ARG
    assert "32 MiB" in lib.rapro_last_error().decode()
    wide = params_for(synth.PAPER_SCALE, 48)
    assert lib.rapro_receive_subframe_noalloc(ctypes.byref(wide), 8, 8, 8, 8, None, None, None, None) == \
        R.RAPRO_ERR_UNSUPPORTED
    half = params_for(synth.PAPER_SCALE, 12)
    half.precision = R.RAPRO_PREC_BF16
    assert lib.rapro_receive_subframe_noalloc(ctypes.byref(half), 8, 8, 8, 8, None, None, None, None) == \
        R.RAPRO_ERR_UNSUPPORTED
    assert "FP32" in lib.rapro_last_error().decode()
    assert lib.rapro_noalloc_status(0, None, None) == R.RAPRO_ERR_INVALID_ARG
