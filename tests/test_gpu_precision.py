"""GPU parity of the precision form's detector half: the Gram and matched filter on the
tensor cores with 16-bit operands (Eq. 22), against the FP64 oracle.

Bars: against the oracle's Gram of the 16-bit-rounded h and y the only difference is the
FP32 accumulation order (products of two 16-bit values are exact in FP32), so 1e-5
norm-wise plus the element-wise bar; against the oracle's Gram of the unrounded inputs the
16-bit rounding itself (2^-7 for BF16, 2^-9 for FP16, norm-wise)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rapro_oracle as O
from paper_1802_05427_gb300 import _build, synth
from paper_1802_05427_gb300 import rapro as R

from _common import assert_parity, params_for

pytestmark = pytest.mark.gpu

FORMS = {"bf16": (False, 2.0 ** -7), "fp16": (True, 2.0 ** -9)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()
    R.lib()
    torch.cuda.set_device(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _channel_and_data(sh, seed):
    """Estimated-channel-like h (the LS + LMMSE output of a subframe) and its data symbols."""
    sf = synth.make_subframe(sh, seed=seed)
    h = np.broadcast_to(np.transpose(sf["H"], (1, 0, 2))[None], (sh.n_slots, sh.K, sh.M, sh.n_sc))
    rng = np.random.default_rng(seed)
    h = h + 0.05 * (rng.standard_normal(h.shape) + 1j * rng.standard_normal(h.shape))
    return synth.as_c64(h), synth.as_c64(sf["y_data"])


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("dims", [(128, 12, 1200, 6), (20, 5, 100, 3), (16, 16, 40, 12), (8, 1, 16, 1),
                                  (33, 7, 58, 6)])
def test_gram_tc_parity(dims, form):
    M, K, N, D = dims
    sh = synth.SubframeShape(M=M, K=K, n_sc=N, n_fft=max(128, 1 << int(np.ceil(np.log2(N)))),
                             n_data_per_slot=D, snr_db=15.0, qam_bits=4)
    h, y = _channel_and_data(sh, 31)
    fp16, tol16 = FORMS[form]
    plan = R.Plan(params_for(sh, 12 if N % 12 == 0 else 4))
    g = torch.empty((sh.n_slots, N, K, K + D), dtype=torch.complex64, device="cuda")
    R.rapro_gram_tc(plan, _dev(h), _dev(y), g, fp16=fp16)
    got = _host(g)
    assert plan.device_status() == 0
    plan.close()
    fmt = "fp16" if fp16 else "bf16"
    A_r, z_r = O.gram_matched_filter(O.round_half(h, fmt), O.round_half(y, fmt), sh.sigma2, D)
    want_r = np.concatenate([A_r, z_r], axis=-1)               # [T][N][K][K + D]
    assert_parity(got, want_r, (1, 2, 3), 1e-5, what=f"{form} vs rounded-input Gram")
    A, z = O.gram_matched_filter(h, y, sh.sigma2, D)
    e, _ = assert_parity(got, np.concatenate([A, z], axis=-1), (1, 2, 3), tol16, what=f"{form} vs exact Gram")
    assert e > 1e-6                                            # the operands really are 16-bit


def test_gram_tc_rejects_what_its_boxes_cannot_read():
    sh = synth.SubframeShape(M=8, K=2, n_sc=75, n_fft=128, qam_bits=2)
    plan = R.Plan(params_for(sh, 5))
    h = torch.zeros(plan.shapes()["h"], dtype=torch.complex64, device="cuda")
    y = torch.zeros(plan.shapes()["y_data"], dtype=torch.complex64, device="cuda")
    g = torch.empty((2, 75, 2, 2 + plan.D), dtype=torch.complex64, device="cuda")
    with pytest.raises(R.RaproError) as e:                      # odd n_sc: no TMA box
        R.rapro_gram_tc(plan, h, y, g)
    assert e.value.status == R.RAPRO_ERR_UNSUPPORTED
    plan.close()


def _detect(plan, h, y, sh):
    s = plan.shapes()
    x = torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda")
    lab = torch.empty(s["labels"], dtype=torch.uint8, device="cuda")
    llr = torch.empty(s["llr"], dtype=torch.float32, device="cuda")
    info = torch.full(s["info"], -7, dtype=torch.int32, device="cuda")
    R.rapro_mmse_detect(plan, _dev(h), _dev(y), x, lab, llr, info)
    return _host(x), _host(lab), _host(llr), _host(info)


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("dims", [(128, 12, 1200, 6, 25.0, 6), (20, 5, 100, 3, 15.0, 4), (16, 16, 40, 12, 20.0, 6),
                                  (33, 7, 58, 6, 10.0, 2), (8, 1, 16, 1, 5.0, 2)])
def test_refined_detector_matches_the_oracle_refinement(dims, form):
    """The precision form's detector (tensor-core Gram of 16-bit operands, FP32 Cholesky, one
    FP32 refinement step) against the oracle's refinement of the same rounded system: the
    FP32 bar; against the exact MMSE output: far inside the unrefined 16-bit error."""
    M, K, N, D, snr, q = dims
    sh = synth.SubframeShape(M=M, K=K, n_sc=N, n_fft=max(128, 1 << int(np.ceil(np.log2(N)))),
                             n_data_per_slot=D, snr_db=snr, qam_bits=q)
    h, y = _channel_and_data(sh, 41)
    fp16, _ = FORMS[form]
    # the 16-bit forms filter on the tensor cores: an even sub-block dividing n_sc
    p = params_for(sh, 12 if N % 12 == 0 else (4 if N % 4 == 0 else 2))
    p.precision = R.RAPRO_PREC_FP16 if fp16 else R.RAPRO_PREC_BF16
    plan = R.Plan(p)
    x, lab, llr, info = _detect(plan, h, y, sh)
    assert plan.device_status() == 0
    plan.close()
    assert (info == 0).all()
    fmt = "fp16" if fp16 else "bf16"
    A_low, z_low = O.gram_matched_filter(O.round_half(h, fmt), O.round_half(y, fmt), sh.sigma2, D)
    x1, s1 = O.refined_mmse_detect(h, y, sh.sigma2, D, A_low, z_low)
    assert_parity(x, x1, (2,), 1e-5, what=f"{form} refined vs oracle refinement")
    x_exact, _ = O.mmse_detect(h, y, sh.sigma2, D)
    x0 = np.empty_like(x_exact)
    for t in range(sh.n_slots):
        x0[t * D:(t + 1) * D] = np.transpose(np.linalg.solve(A_low[t], z_low[t]), (2, 1, 0))
    from _common import rel_err_per
    e1, e0 = rel_err_per(x, x_exact, (2,)).max(), rel_err_per(x0, x_exact, (2,)).max()
    assert e1 < 0.1 * e0 and e1 < 2e-3, (e1, e0)
    # hard decisions of the refined output against the oracle's, away from decision boundaries
    xh, _ = O.unbias(x1, s1, D)
    safe = O.boundary_margin(xh, q) > 1e-3
    np.testing.assert_array_equal(lab[safe], O.hard_decision(xh, q)[safe])


def test_sixteen_bit_plans_can_take_the_fp32_detector():
    """RAPRO_DET_FP32 on a BF16 plan: the FP32 Gram and matched filter (Eq. 22) at the FP32
    bar against the oracle; the form is rejected for an FP32 plan and for unknown values."""
    sh = synth.SubframeShape(M=24, K=6, n_sc=96, n_fft=128, n_data_per_slot=6, snr_db=15.0, qam_bits=4)
    h, y = _channel_and_data(sh, 47)
    p = params_for(sh, 8)
    p.precision = R.RAPRO_PREC_BF16
    plan = R.Plan(p)
    R.rapro_plan_set_detector_form(plan, R.RAPRO_DET_FP32)
    x, lab, llr, info = _detect(plan, h, y, sh)
    assert plan.device_status() == 0 and (info == 0).all()
    x_o, _ = O.mmse_detect(h.astype(np.complex128), y.astype(np.complex128), sh.sigma2, sh.n_data_per_slot)
    assert_parity(x, x_o, (2,), 1e-5, what="FP32 detector of a BF16 plan")
    with pytest.raises(R.RaproError) as e:
        R.rapro_plan_set_detector_form(plan, 7)
    assert e.value.status == R.RAPRO_ERR_INVALID_ARG
    plan.close()
    with R.Plan(params_for(sh, 8)) as p32:
        with pytest.raises(R.RaproError) as e:
            R.rapro_plan_set_detector_form(p32, R.RAPRO_DET_FP32)
        assert e.value.status == R.RAPRO_ERR_UNSUPPORTED
