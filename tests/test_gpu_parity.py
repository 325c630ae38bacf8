"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Both sides read the same complex64 inputs.  Bars (FP32 device arithmetic):
  * channel estimates and equalised symbols: norm-wise relative error <= 1e-5 per
    (slot, user) resp. (data symbol, user);
  * hard decisions identical wherever the oracle's unbiased symbol is farther than
    1e-4 d_min/2 from a decision boundary; elsewhere the device label must still be a
    nearest point within that tolerance;
  * LLRs within 1e-4 relative plus the absolute error that a 1e-5 relative error of
    x^ produces through the piecewise-linear max-log metric: 4 (2^m - 1) 1e-5 |x^|_s / (nu s)
    (s = lattice scale, m bits per dimension);
  * info == 0 unless a pivot is not positive and finite.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rapro_oracle as O
from oracle import rapro_grad_oracle as G
from paper_1802_05427_gb300 import _build, synth
from paper_1802_05427_gb300 import rapro as R

from _common import assert_parity, params_for, oracle_r, rel_err_per

pytestmark = pytest.mark.gpu

TOL = 1e-5
MARGIN = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()
    R.lib()
    torch.cuda.set_device(0)


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda") if dtype is None else t.to("cuda", dtype=dtype)


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _inputs(sh, seed):
    sf = synth.make_subframe(sh, seed=seed)
    return sf, {k: synth.as_c64(sf[k]) for k in ("y_pilot", "pilots", "y_data")}


def gpu_receive(sh, c64, B, pdp="exp", h_out=True):
    plan = R.Plan(params_for(sh, B, pdp=pdp))
    s = plan.shapes()
    yp, pil, yd = _dev(c64["y_pilot"]), _dev(c64["pilots"]), _dev(c64["y_data"])
    x = torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda")
    lab = torch.empty(s["labels"], dtype=torch.uint8, device="cuda")
    llr = torch.empty(s["llr"], dtype=torch.float32, device="cuda")
    info = torch.full(s["info"], -7, dtype=torch.int32, device="cuda")
    h = torch.empty(s["h"], dtype=torch.complex64, device="cuda") if h_out else None
    R.rapro_receive_subframe(plan, yp, pil, yd, x, lab, llr, info, h_out=h)
    out = dict(x_eq=_host(x), labels=_host(lab), llr=_host(llr), info=_host(info))
    if h_out:
        out["h"] = _host(h)
    assert plan.device_status() == 0
    plan.close()
    return out


def oracle_receive(sh, c64, B, pdp="exp"):
    return O.receive_subframe(c64["y_pilot"].astype(np.complex128), c64["pilots"].astype(np.complex128),
                              c64["y_data"].astype(np.complex128), B=B, sigma2=sh.sigma2,
                              r=oracle_r(sh, pdp), n_data_per_slot=sh.n_data_per_slot, q=sh.qam_bits)


def check_detection(g, o, q):
    assert_parity(g["x_eq"], o["x_eq"], (2,), TOL, what="x_eq")
    margin = O.boundary_margin(o["xhat"], q)
    safe = margin > MARGIN
    bad = (g["labels"] != o["labels"]) & safe
    assert not bad.any(), f"{bad.sum()} hard decisions differ away from boundaries"
    # near a boundary the device label must still be a nearest point (within tolerance)
    pts = O.constellation(q)
    near = ~safe
    if near.any():
        xh = o["xhat"][near]
        dmin = np.min(np.abs(xh[:, None] - pts[None]) ** 2, axis=1)
        dg = np.abs(xh - pts[g["labels"][near].astype(int)]) ** 2
        assert np.all(dg - dmin <= 1e-6 * (1 + np.abs(xh) ** 2))
    assert near.mean() < 1e-3
    m = q // 2
    s = np.sqrt(2.0 * (4 ** m - 1) / 3.0)
    xmag = np.maximum(1.0, np.abs(o["xhat"]))[..., None]
    tol = 1e-4 * np.abs(o["llr"]) + 4 * (2 ** m - 1) * 10 * TOL * xmag / (o["nu"][..., None] * s)
    err = np.abs(g["llr"] - o["llr"])
    assert np.all(err <= tol), f"llr worst excess {np.max(err - tol):.3g}"
    # LLR signs agree with the device's own hard bits
    bits = (g["labels"][..., None] >> (q - 1 - np.arange(q))) & 1
    nz = np.abs(g["llr"]) > 0
    assert np.all((g["llr"][nz] > 0) == (bits[nz] == 0))


# ------------------------------------------------------------------------ LS
@pytest.mark.parametrize("dims", [(8, 2, 72), (20, 5, 100), (3, 1, 75), (128, 12, 1200)])
def test_ls_parity(dims):
    M, K, N = dims
    sh = synth.SubframeShape(M=M, K=K, n_sc=N, n_fft=max(128, 2 * N), qam_bits=2)
    sf, c64 = _inputs(sh, 1)
    plan = R.Plan(params_for(sh, min(12, N)))
    h = torch.empty(plan.shapes()["h"], dtype=torch.complex64, device="cuda")
    R.rapro_ce_ls(plan, _dev(c64["y_pilot"]), _dev(c64["pilots"]), h)
    ref = O.ls_estimate(c64["y_pilot"].astype(np.complex128), c64["pilots"].astype(np.complex128))
    assert_parity(_host(h), ref, (2, 3), 1e-6)


# --------------------------------------------------------------------- LMMSE
LMMSE_CASES = [
    # M, K, N, n_fft, B
    (8, 2, 72, 128, 12), (8, 2, 72, 128, 1), (8, 2, 72, 128, 72), (5, 3, 100, 256, 12),
    (5, 3, 100, 256, 7), (4, 2, 130, 256, 33), (4, 2, 130, 256, 48), (4, 2, 200, 256, 100),
    (6, 2, 75, 128, 16), (3, 2, 90, 128, 24), (3, 2, 96, 128, 32), (2, 1, 64, 128, 4),
    (128, 12, 1200, 2048, 12), (128, 12, 1200, 2048, 48), (128, 12, 1200, 2048, 100),
    (128, 12, 1200, 2048, 1200),
]


@pytest.mark.parametrize("case", LMMSE_CASES)
def test_lmmse_parity(case):
    M, K, N, nfft, B = case
    sh = synth.SubframeShape(M=M, K=K, n_sc=N, n_fft=nfft, n_taps=24 if nfft >= 2048 else 6,
                             tau_rms=8.0 if nfft >= 2048 else 4.0, snr_db=10.0, qam_bits=2)
    sf, c64 = _inputs(sh, 2)
    h_ls = synth.as_c64(O.ls_estimate(c64["y_pilot"], c64["pilots"]))
    plan = R.Plan(params_for(sh, B))
    h = torch.empty(plan.shapes()["h"], dtype=torch.complex64, device="cuda")
    R.rapro_ce_lmmse_subblock(plan, _dev(h_ls), h)
    ref = O.subblock_lmmse(h_ls.astype(np.complex128), B, oracle_r(sh), sh.sigma2)
    assert_parity(_host(h), ref, (2, 3), TOL)


@pytest.mark.parametrize("B", [12, 40])
def test_lmmse_weight_override(B):
    """w_override: one W per block (here random), applied block by block (Eq. 12)."""
    sh = synth.SubframeShape(M=6, K=2, n_sc=100, n_fft=256, qam_bits=2)
    sf, c64 = _inputs(sh, 3)
    h_ls = synth.as_c64(O.ls_estimate(c64["y_pilot"], c64["pilots"]))
    plan = R.Plan(params_for(sh, B))
    rng = np.random.default_rng(5)
    weights, flat = [], []
    for b0 in range(0, sh.n_sc, B):
        n = min(B, sh.n_sc - b0)
        W = synth.as_c64((rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / n)
        weights.append((b0, W.astype(np.complex128)))
        flat.append(W.ravel())
    h = torch.empty(plan.shapes()["h"], dtype=torch.complex64, device="cuda")
    R.rapro_ce_lmmse_subblock(plan, _dev(h_ls), h, w_override=_dev(np.concatenate(flat)))
    ref = O.subblock_lmmse(h_ls.astype(np.complex128), B, None, None, weights=weights)
    assert_parity(_host(h), ref, (2, 3), TOL)


LS_LMMSE_CASES = [
    # M, K, N, n_fft, B: even B <= 16 dividing N runs on the tensor cores (tiles ragged in the
    # antennas and in the blocks, several tiles per CTA); the rest on the FP32 cores
    (8, 2, 72, 128, 12), (5, 3, 100, 256, 10), (6, 2, 96, 128, 16), (3, 2, 90, 128, 6),
    (2, 1, 64, 128, 2), (4, 3, 120, 256, 8), (7, 2, 84, 128, 14), (128, 12, 1200, 2048, 4),
    (128, 12, 1200, 2048, 12), (128, 12, 1200, 2048, 16), (5, 3, 100, 256, 12), (5, 3, 100, 256, 7),
    (128, 12, 1200, 2048, 48), (130, 1, 48, 128, 12), (200, 2, 32, 128, 16),
]


TCG_CASES = [
    # M, K, N, n_fft, B: even B > 16 dividing N (the tensor-core GEMM); rows not a multiple
    # of the 128-row tile, K chunks of 16 subcarriers running past the block (B = 18, 100),
    # one block (the full LMMSE, B = N), several output tiles (2B > 128)
    (20, 3, 72, 128, 18), (50, 5, 96, 256, 24), (7, 2, 96, 128, 48), (16, 2, 200, 256, 100),
    (9, 1, 120, 256, 120), (33, 4, 240, 512, 80),
]


@pytest.mark.parametrize("case", TCG_CASES)
def test_tensor_core_gemm_estimator_parity(case):
    """The large-block filter on tcgen05 (three TF32 passes), with LS fused (rapro_ce_ls_lmmse)
    and on a given h_ls (rapro_ce_lmmse_subblock), against the oracle; the built-in choice and
    the explicit variant agree, and the FP32 tiled kernel agrees with both."""
    M, K, N, nfft, B = case
    sh = synth.SubframeShape(M=M, K=K, n_sc=N, n_fft=nfft, snr_db=12.0, qam_bits=2)
    sf, c64 = _inputs(sh, 31)
    h_ls = O.ls_estimate(c64["y_pilot"].astype(np.complex128), c64["pilots"].astype(np.complex128))
    ref = O.subblock_lmmse(h_ls, B, oracle_r(sh), sh.sigma2)
    plan = R.Plan(params_for(sh, B))
    shp = plan.shapes()["h"]
    yp, pil, hl = _dev(c64["y_pilot"]), _dev(c64["pilots"]), _dev(synth.as_c64(h_ls))
    outs = {}
    for ev in (-1, 4, 3):
        R.rapro_plan_set_variant(plan, ev, 1, 1)
        for fused in (True, False):
            h = torch.full(shp, 5.0 + 5j, dtype=torch.complex64, device="cuda")
            if fused:
                R.rapro_ce_ls_lmmse(plan, yp, pil, h)
            else:
                R.rapro_ce_lmmse_subblock(plan, hl, h)
            g = _host(h)
            assert_parity(g, ref, (2, 3), TOL, what=str((ev, fused)))
            outs[(ev, fused)] = g
    assert np.array_equal(outs[(-1, True)], outs[(4, True)])           # the built-in choice is the GEMM
    assert plan.device_status() == 0
    plan.close()


@pytest.mark.parametrize("case", LS_LMMSE_CASES)
def test_ls_lmmse_parity(case):
    """LS (Eq. 9) and the sub-block filter (Eq. 12, 17) in one call, against both oracle steps."""
    M, K, N, nfft, B = case
    sh = synth.SubframeShape(M=M, K=K, n_sc=N, n_fft=nfft, n_taps=24 if nfft >= 2048 else 6,
                             tau_rms=8.0 if nfft >= 2048 else 4.0, snr_db=10.0, qam_bits=2)
    sf, c64 = _inputs(sh, 4)
    plan = R.Plan(params_for(sh, B))
    h = torch.empty(plan.shapes()["h"], dtype=torch.complex64, device="cuda")
    R.rapro_ce_ls_lmmse(plan, _dev(c64["y_pilot"]), _dev(c64["pilots"]), h)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    h_ls = O.ls_estimate(c64["y_pilot"].astype(np.complex128), c64["pilots"].astype(np.complex128))
    ref = O.subblock_lmmse(h_ls, B, oracle_r(sh), sh.sigma2)
    assert_parity(_host(h), ref, (2, 3), TOL)


# ----------------------------------------------------------------- detection
DETECT_CASES = [
    # M, K, N, D, q
    (8, 2, 72, 6, 2), (20, 5, 100, 6, 4), (128, 12, 1200, 6, 4), (64, 16, 96, 12, 6),
    (1, 1, 40, 6, 2), (3, 3, 33, 6, 2), (16, 7, 75, 5, 6), (36, 12, 48, 1, 4), (9, 4, 16, 12, 2),
]


@pytest.mark.parametrize("case", DETECT_CASES)
def test_detect_parity(case):
    M, K, N, D, q = case
    sh = synth.SubframeShape(M=M, K=K, n_sc=N, n_fft=max(128, 2 * N), qam_bits=q, n_data_per_slot=D,
                             snr_db=15.0)
    sf, c64 = _inputs(sh, 4)
    h = synth.as_c64(O.subblock_lmmse(O.ls_estimate(c64["y_pilot"], c64["pilots"]), min(12, N),
                                      oracle_r(sh), sh.sigma2))
    plan = R.Plan(params_for(sh, min(12, N)))
    s = plan.shapes()
    x = torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda")
    lab = torch.empty(s["labels"], dtype=torch.uint8, device="cuda")
    llr = torch.empty(s["llr"], dtype=torch.float32, device="cuda")
    info = torch.full(s["info"], -1, dtype=torch.int32, device="cuda")
    R.rapro_mmse_detect(plan, _dev(h), _dev(c64["y_data"]), x, lab, llr, info)
    x_o, s_o = O.mmse_detect(h.astype(np.complex128), c64["y_data"].astype(np.complex128), sh.sigma2, D)
    xhat, nu = O.unbias(x_o, s_o, D)
    o = dict(x_eq=x_o, xhat=xhat, nu=nu, labels=O.hard_decision(xhat, q), llr=O.maxlog_llr(xhat, nu, q))
    g = dict(x_eq=_host(x), labels=_host(lab), llr=_host(llr))
    check_detection(g, o, q)
    assert np.all(_host(info) == 0)
    assert plan.device_status() == 0


def test_detect_optional_outputs_may_be_null():
    sh = synth.SubframeShape(M=8, K=3, n_sc=40, n_fft=128, qam_bits=4)
    sf, c64 = _inputs(sh, 6)
    h = synth.as_c64(O.ls_estimate(c64["y_pilot"], c64["pilots"]))
    plan = R.Plan(params_for(sh, 8))
    x = torch.empty(plan.shapes()["x_eq"], dtype=torch.complex64, device="cuda")
    R.rapro_mmse_detect(plan, _dev(h), _dev(c64["y_data"]), x)
    x_o, _ = O.mmse_detect(h.astype(np.complex128), c64["y_data"].astype(np.complex128), sh.sigma2, 6)
    assert_parity(_host(x), x_o, (2,), TOL)


def test_nan_subcarrier_sets_info_and_spares_the_rest():
    """A non-finite channel estimate makes pivot 1 fail on that subcarrier only."""
    sh = synth.SubframeShape(M=8, K=3, n_sc=40, n_fft=128, qam_bits=2)
    sf, c64 = _inputs(sh, 7)
    h = synth.as_c64(O.ls_estimate(c64["y_pilot"], c64["pilots"]))
    h[1, :, :, 17] = np.nan
    plan = R.Plan(params_for(sh, 8))
    s = plan.shapes()
    x = torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda")
    info = torch.full(s["info"], -1, dtype=torch.int32, device="cuda")
    R.rapro_mmse_detect(plan, _dev(h), _dev(c64["y_data"]), x, info=info)
    inf_h, x_h = _host(info), _host(x)
    assert inf_h[1, 17] == 1
    assert np.count_nonzero(inf_h) == 1
    assert np.isnan(x_h[6:12, :, 17]).all()
    good = np.ones(sh.n_sc, bool)
    good[17] = False
    x_o, _ = O.mmse_detect(h[:1].astype(np.complex128), c64["y_data"][:6].astype(np.complex128), sh.sigma2, 6)
    assert_parity(x_h[:6], x_o, (2,), TOL)
    assert np.isfinite(x_h[6:12][..., good]).all()


# ------------------------------------------------------------- whole receive
RECEIVE_CASES = [
    ("tiny", synth.TINY, 12, 0), ("ragged", synth.SubframeShape(M=20, K=5, n_sc=100, n_fft=256, n_taps=6,
                                                                 tau_rms=4.0, snr_db=12.0, qam_bits=4), 12, 1),
    ("odd_nsc", synth.SubframeShape(M=12, K=4, n_sc=75, n_fft=128, snr_db=8.0, qam_bits=2), 10, 2),
]


@pytest.mark.parametrize("name,sh,B,seed", RECEIVE_CASES, ids=[c[0] for c in RECEIVE_CASES])
def test_receive_subframe_parity_small(name, sh, B, seed):
    sf, c64 = _inputs(sh, synth.SEED_BASE + seed)
    g = gpu_receive(sh, c64, B)
    o = oracle_receive(sh, c64, B)
    assert_parity(g["h"], o["h"], (2, 3), TOL)
    check_detection(g, o, sh.qam_bits)
    assert np.all(g["info"] == 0)


@pytest.mark.parametrize("snr", [0.0, 10.0, 20.0])
@pytest.mark.parametrize("B", [12, 48, 100, 1200])
def test_receive_subframe_parity_paper_scale(B, snr):
    """M = 128, K = 12, 1200 subcarriers, 16-QAM, 24-tap exponential PDP (the headline
    workload), every output compared in full."""
    sh = synth.SubframeShape(**{**synth.PAPER_SCALE.__dict__, "snr_db": snr})
    sf, c64 = _inputs(sh, synth.SEED_BASE + 1)
    g = gpu_receive(sh, c64, B)
    o = oracle_receive(sh, c64, B)
    assert_parity(g["h"], o["h"], (2, 3), TOL)
    check_detection(g, o, sh.qam_bits)
    assert np.all(g["info"] == 0)


def test_receive_without_h_out_and_uniform_L_model():
    sh = synth.SubframeShape(M=16, K=4, n_sc=96, n_fft=256, snr_db=15.0, qam_bits=6)
    sf, c64 = _inputs(sh, 11)
    g = gpu_receive(sh, c64, 12, pdp="uniform_L", h_out=False)
    o = oracle_receive(sh, c64, 12, pdp="uniform_L")
    check_detection(g, o, sh.qam_bits)


# ------------------------------------------ fused receive form (one kernel per subframe)
FUSED_CASES = [
    # name, shape, B: block sizes that give pilot boxes of 12 .. 30 subcarriers, tail blocks,
    # n_sc not a multiple of the 16-subcarrier tile, antennas not a multiple of the 8-antenna
    # chunk, 1..16 users (16: several users per half-warp), 12 data symbols per slot
    ("tiny_B12", synth.TINY, 12),
    ("B2", synth.SubframeShape(M=9, K=3, n_sc=50, n_fft=128, qam_bits=2), 2),
    ("B4_K1", synth.SubframeShape(M=16, K=1, n_sc=36, n_fft=64, qam_bits=4), 4),
    ("B6_tail", synth.SubframeShape(M=20, K=5, n_sc=100, n_fft=256, snr_db=12.0, qam_bits=4), 6),
    ("B8", synth.SubframeShape(M=24, K=8, n_sc=120, n_fft=256, qam_bits=6), 8),
    ("B10_tail", synth.SubframeShape(M=13, K=6, n_sc=104, n_fft=256, qam_bits=4), 10),
    ("B12_tail_K16", synth.SubframeShape(M=40, K=16, n_sc=206, n_fft=512, n_taps=8, tau_rms=5.0,
                                         snr_db=20.0, qam_bits=4), 12),
    ("B14_D12", synth.SubframeShape(M=17, K=12, n_sc=140, n_fft=256, qam_bits=2, n_data_per_slot=12), 14),
    ("B16_K16_D12", synth.SubframeShape(M=32, K=16, n_sc=96, n_fft=128, qam_bits=6, n_data_per_slot=12,
                                        snr_db=25.0), 16),
]


@pytest.mark.parametrize("name,sh,B", FUSED_CASES, ids=[c[0] for c in FUSED_CASES])
def test_fused_receive_matches_the_oracle(name, sh, B):
    """Eq. 9, 12, 20-22 in one kernel: h (when asked for), x~, labels, LLRs and info as
    the oracle; without h_out the same outputs and nothing else written."""
    sf, c64 = _inputs(sh, synth.SEED_BASE + 40)
    o = oracle_receive(sh, c64, B)
    plan = R.Plan(params_for(sh, B))
    s = plan.shapes()
    yp, pil, yd = _dev(c64["y_pilot"]), _dev(c64["pilots"]), _dev(c64["y_data"])
    assert not R.rapro_receive_is_fused(plan, yp, yd)            # the default form is split
    R.rapro_plan_set_receive_form(plan, R.RAPRO_RECV_FUSED)
    assert R.rapro_receive_is_fused(plan, yp, yd)
    for with_h in (True, False):
        x = torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda")
        lab = torch.empty(s["labels"], dtype=torch.uint8, device="cuda")
        llr = torch.empty(s["llr"], dtype=torch.float32, device="cuda")
        info = torch.full(s["info"], -7, dtype=torch.int32, device="cuda")
        h = torch.full(s["h"], 3.0 + 1j, dtype=torch.complex64, device="cuda") if with_h else None
        R.rapro_receive_subframe(plan, yp, pil, yd, x, lab, llr, info, h_out=h)
        g = dict(x_eq=_host(x), labels=_host(lab), llr=_host(llr), info=_host(info))
        if with_h:
            assert_parity(_host(h), o["h"], (2, 3), TOL)
        check_detection(g, o, sh.qam_bits)
        assert np.all(g["info"] == 0)
    assert plan.device_status() == 0
    plan.close()


def test_fused_and_split_forms_agree_and_the_form_is_selectable():
    sh = synth.SubframeShape(M=32, K=12, n_sc=192, n_fft=256, snr_db=15.0, qam_bits=4)
    sf, c64 = _inputs(sh, synth.SEED_BASE + 41)
    o = oracle_receive(sh, c64, 12)
    plan = R.Plan(params_for(sh, 12))
    s = plan.shapes()
    yp, pil, yd = _dev(c64["y_pilot"]), _dev(c64["pilots"]), _dev(c64["y_data"])
    outs = {}
    for form in (R.RAPRO_RECV_SPLIT, R.RAPRO_RECV_FUSED):
        R.rapro_plan_set_receive_form(plan, form)
        assert R.rapro_receive_is_fused(plan, yp, yd) == (form == R.RAPRO_RECV_FUSED)
        x = torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda")
        lab = torch.empty(s["labels"], dtype=torch.uint8, device="cuda")
        R.rapro_receive_subframe(plan, yp, pil, yd, x, lab)
        outs[form] = (_host(x), _host(lab))
        assert_parity(outs[form][0], o["x_eq"], (2,), TOL)
    # both forms round differently (LS folded into the weights), but only in the last bits
    assert_parity(outs[0][0], outs[1][0], (2,), 2 * TOL)
    assert (outs[0][1] == outs[1][1]).mean() > 0.999
    with pytest.raises(R.RaproError):
        R.rapro_plan_set_receive_form(plan, 7)
    plan.close()


def test_fused_form_applies_only_where_its_rules_hold():
    """Odd n_sc, B > 16, odd B, BF16 plans, comb plans and unaligned arrays take the
    two-kernel form (and still match the oracle where it is run here)."""
    sh = synth.SubframeShape(M=16, K=4, n_sc=96, n_fft=128, qam_bits=2)
    sf, c64 = _inputs(sh, synth.SEED_BASE + 42)
    yp, yd = _dev(c64["y_pilot"]), _dev(c64["y_data"])
    def fused_plan(p):
        plan = R.Plan(p)
        R.rapro_plan_set_receive_form(plan, R.RAPRO_RECV_FUSED)
        return plan

    for B, ok in ((12, True), (48, False), (9, False), (16, True)):
        with fused_plan(params_for(sh, B)) as plan:
            assert R.rapro_receive_is_fused(plan, yp, yd) == ok, B
    p = params_for(sh, 12)
    p.precision = R.RAPRO_PREC_BF16
    with fused_plan(p) as plan:
        assert not R.rapro_receive_is_fused(plan, yp, yd)
    sh_odd = synth.SubframeShape(M=8, K=2, n_sc=75, n_fft=128, qam_bits=2)
    sfo, co = _inputs(sh_odd, 3)
    with fused_plan(params_for(sh_odd, 10)) as plan:
        assert not R.rapro_receive_is_fused(plan, _dev(co["y_pilot"]), _dev(co["y_data"]))
    # an 8-byte offset view: same values, not 16-byte aligned
    with fused_plan(params_for(sh, 12)) as plan:
        s = plan.shapes()
        buf = torch.empty(int(np.prod(s["y_pilot"])) + 1, dtype=torch.complex64, device="cuda")
        ypu = buf[1:].view(s["y_pilot"])
        ypu.copy_(yp)
        assert not R.rapro_receive_is_fused(plan, ypu, yd)
        x = torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda")
        R.rapro_receive_subframe(plan, ypu, _dev(c64["pilots"]), yd, x)
        o = oracle_receive(sh, c64, 12)
        assert_parity(_host(x), o["x_eq"], (2,), TOL)


def test_invalid_pointers_are_rejected_without_launch():
    sh = synth.TINY
    plan = R.Plan(params_for(sh, 12))
    lib = R.lib()
    assert lib.rapro_ce_ls(plan.handle, None, None, None, None) == R.RAPRO_ERR_INVALID_ARG
    assert lib.rapro_mmse_detect(plan.handle, None, None, None, None, None, None, None) == R.RAPRO_ERR_INVALID_ARG
    assert lib.rapro_receive_subframe(None, None, None, None, None, None, None, None, None, None) == \
        R.RAPRO_ERR_INVALID_ARG
    x = torch.empty(plan.shapes()["h"], dtype=torch.complex64, device="cuda")
    assert lib.rapro_ce_lmmse_subblock(plan.handle, x.data_ptr(), None, x.data_ptr(), None) == \
        R.RAPRO_ERR_INVALID_ARG
    assert plan.device_status() == 0


# ------------------------------------------------------- comb pilots (Sec. II, IV-B)
COMB_METHODS = {R.RAPRO_COMB_3W: O.COMB_3W, R.RAPRO_COMB_SW: O.COMB_SW, R.RAPRO_COMB_INTERP3: O.COMB_INTERP3}
COMB_CASES = [
    # name, shape, comb spacing S
    ("tiny", synth.SubframeShape(M=8, K=2, n_sc=72, n_fft=128, qam_bits=2), 6),
    ("ragged_antennas", synth.SubframeShape(M=13, K=4, n_sc=96, n_fft=128, n_taps=5, tau_rms=3.0, qam_bits=2), 6),
    ("spacing15", synth.SubframeShape(M=5, K=3, n_sc=240, n_fft=512, qam_bits=4), 15),
    ("paper_scale", synth.PAPER_SCALE, 12),
]


def comb_params(sh, S, method):
    p = params_for(sh, 1)
    p.pilot_layout, p.comb_spacing, p.comb_method, p.subblock = R.RAPRO_PILOT_COMB, S, method, 0
    return p


def oracle_comb_h(sh, c64, S, method):
    h_ls = O.comb_ls(c64["y_pilot"].astype(np.complex128), c64["pilots"].astype(np.complex128), sh.K, S)
    if method == R.RAPRO_COMB_INTERP3:
        return O.comb_interp3_ls(h_ls, S, sh.n_sc)
    return O.comb_lmmse(h_ls, COMB_METHODS[method], S, sh.n_sc, oracle_r(sh), sh.sigma2)


@pytest.mark.parametrize("method", list(COMB_METHODS), ids=["3W", "SW", "interp3"])
@pytest.mark.parametrize("name,sh,S", COMB_CASES, ids=[c[0] for c in COMB_CASES])
def test_comb_estimate_parity(name, sh, S, method):
    """rapro_ce_comb against the oracle: LS on each user's tones, the groups of Tables I-II
    with their weights, interpolation and zero-order hold, for every user and subcarrier."""
    sf = synth.make_comb_subframe(sh, seed=synth.SEED_BASE + 30, S=S)
    c64 = {k: synth.as_c64(sf[k]) for k in ("y_pilot", "pilots", "y_data")}
    plan = R.Plan(comb_params(sh, S, method))
    h = torch.empty(plan.shapes()["h"], dtype=torch.complex64, device="cuda")
    R.rapro_ce_comb(plan, _dev(c64["y_pilot"]), _dev(c64["pilots"]), h)
    ref = oracle_comb_h(sh, c64, S, method)
    assert_parity(_host(h), ref, (2, 3), TOL)


@pytest.mark.parametrize("method", list(COMB_METHODS), ids=["3W", "SW", "interp3"])
def test_comb_receive_subframe_parity(method):
    """The whole comb-pilot receive (estimate, then the MMSE detector) against the oracle."""
    sh = synth.SubframeShape(M=32, K=8, n_sc=600, n_fft=1024, n_taps=6, tau_rms=3.0, snr_db=18.0, qam_bits=4)
    S = 12
    sf = synth.make_comb_subframe(sh, seed=synth.SEED_BASE + 31, S=S)
    c64 = {k: synth.as_c64(sf[k]) for k in ("y_pilot", "pilots", "y_data")}
    plan = R.Plan(comb_params(sh, S, method))
    s = plan.shapes()
    x = torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda")
    lab = torch.empty(s["labels"], dtype=torch.uint8, device="cuda")
    llr = torch.empty(s["llr"], dtype=torch.float32, device="cuda")
    info = torch.full(s["info"], -7, dtype=torch.int32, device="cuda")
    h = torch.empty(s["h"], dtype=torch.complex64, device="cuda")
    R.rapro_receive_subframe(plan, _dev(c64["y_pilot"]), _dev(c64["pilots"]), _dev(c64["y_data"]), x, lab, llr,
                             info, h_out=h)
    o = O.comb_receive_subframe(c64["y_pilot"].astype(np.complex128), c64["pilots"].astype(np.complex128),
                                c64["y_data"].astype(np.complex128), K=sh.K, S=S, method=COMB_METHODS[method],
                                sigma2=sh.sigma2, r=oracle_r(sh), n_data_per_slot=sh.n_data_per_slot,
                                q=sh.qam_bits)
    assert_parity(_host(h), o["h"], (2, 3), TOL)
    assert (_host(info) == 0).all()
    check_detection(dict(x_eq=_host(x), labels=_host(lab), llr=_host(llr)), o, sh.qam_bits)


def test_comb_and_orthogonal_plans_reject_each_others_estimators():
    sh = synth.TINY
    comb = R.Plan(comb_params(sh, 6, R.RAPRO_COMB_SW))
    orth = R.Plan(params_for(sh, 12))
    sc, so = comb.shapes(), orth.shapes()
    h = torch.empty(sc["h"], dtype=torch.complex64, device="cuda")
    with pytest.raises(R.RaproError) as e:
        R.rapro_ce_ls_lmmse(comb, torch.zeros(sc["y_pilot"], dtype=torch.complex64, device="cuda"),
                            torch.zeros(sc["pilots"], dtype=torch.complex64, device="cuda"), h)
    assert e.value.status == R.RAPRO_ERR_UNSUPPORTED
    with pytest.raises(R.RaproError) as e:
        R.rapro_ce_comb(orth, torch.zeros(so["y_pilot"], dtype=torch.complex64, device="cuda"),
                        torch.zeros(so["pilots"], dtype=torch.complex64, device="cuda"), h)
    assert e.value.status == R.RAPRO_ERR_UNSUPPORTED


# --------------------------------------------- precision form (BF16 tensor cores)
# One BF16 pass rounds the LS estimate and W to 8 significant bits (unit roundoff 2^-9
# each) and accumulates in FP32: per output |err| <= sum_j |W_ij| |x_j| (2^-8 + 2^-16), so
# norm-wise about 2^-8 / sqrt(3) for random signs; the bound below is 2^-7.
TOL_BF16 = 2.0 ** -7
# FP16 keeps 11 significant bits (unit roundoff 2^-11): the same argument gives 2^-9.
TOL_FP16 = 2.0 ** -9
HALF_FORMS = {"bf16": (R.RAPRO_PREC_BF16, TOL_BF16), "fp16": (R.RAPRO_PREC_FP16, TOL_FP16)}


@pytest.mark.parametrize("form", list(HALF_FORMS))
@pytest.mark.parametrize("case", [(8, 2, 72, 128, 12), (5, 3, 100, 256, 10), (6, 2, 96, 128, 16),
                                  (2, 1, 64, 128, 2), (128, 12, 1200, 2048, 12),
                                  # larger blocks: the tensor-core GEMM with 16-bit operands
                                  (20, 3, 72, 128, 18), (7, 2, 96, 128, 48), (16, 2, 200, 256, 100),
                                  (33, 4, 240, 512, 80), (128, 12, 1200, 2048, 1200),
                                  # 256-column tiles: one tile (W resident), a ragged last tile
                                  (9, 2, 256, 512, 128), (11, 3, 600, 1024, 300)])
def test_bf16_estimator_parity(case, form):
    M, K, N, nfft, B = case
    sh = synth.SubframeShape(M=M, K=K, n_sc=N, n_fft=nfft, n_taps=24 if nfft >= 2048 else 6,
                             tau_rms=8.0 if nfft >= 2048 else 4.0, snr_db=10.0, qam_bits=2)
    sf, c64 = _inputs(sh, 5)
    prec, tol = HALF_FORMS[form]
    p = params_for(sh, B)
    p.precision = prec
    plan = R.Plan(p)
    h = torch.empty(plan.shapes()["h"], dtype=torch.complex64, device="cuda")
    R.rapro_ce_ls_lmmse(plan, _dev(c64["y_pilot"]), _dev(c64["pilots"]), h)
    h_ls = O.ls_estimate(c64["y_pilot"].astype(np.complex128), c64["pilots"].astype(np.complex128))
    ref = O.subblock_lmmse(h_ls, B, oracle_r(sh), sh.sigma2)
    e, _ = assert_parity(_host(h), ref, (2, 3), tol, what=form)
    assert e > 1e-5                        # it really is the single 16-bit pass
    if form == "fp16":
        assert e < TOL_BF16 / 4            # and FP16's three extra bits show
    with pytest.raises(R.RaproError):
        R.rapro_ce_lmmse_subblock(plan, _dev(synth.as_c64(h_ls)), h)


@pytest.mark.parametrize("B", [12, 48, 1200])
@pytest.mark.parametrize("form", list(HALF_FORMS))
def test_bf16_form_keeps_nmse_and_evm_within_a_tenth_of_a_db(form, B):
    """Precision forms on the paper-scale shape (64-QAM, 25 dB, several subframes) at small,
    medium and full-LMMSE blocks: channel NMSE and post-detection EVM within 0.1 dB of the
    FP64 oracle's."""
    sh = synth.SubframeShape(**{**synth.PAPER_SCALE.__dict__, "snr_db": 25.0, "qam_bits": 6})
    p = params_for(sh, B)
    p.precision = HALF_FORMS[form][0]
    plan = R.Plan(p)
    s = plan.shapes()
    err_h = err_h_o = pow_h = err_x = err_x_o = pow_x = 0.0
    for i in range(4):
        sf, c64 = _inputs(sh, synth.SEED_BASE + 40 + i)
        x = torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda")
        h = torch.empty(s["h"], dtype=torch.complex64, device="cuda")
        R.rapro_receive_subframe(plan, _dev(c64["y_pilot"]), _dev(c64["pilots"]), _dev(c64["y_data"]), x, h_out=h)
        o = oracle_receive(sh, c64, B)
        H = np.transpose(sf["H"], (1, 0, 2))[None]
        err_h += np.sum(np.abs(_host(h) - H) ** 2)
        err_h_o += np.sum(np.abs(o["h"] - H) ** 2)
        pow_h += 2 * np.sum(np.abs(H) ** 2)
        mu = 1.0 - o["s"]                                     # the oracle's unbiasing for both
        T, D = sh.n_slots, sh.n_data_per_slot
        xh = _host(x) / np.repeat(mu, D, axis=0)
        err_x += np.sum(np.abs(xh - sf["x"]) ** 2)
        err_x_o += np.sum(np.abs(o["xhat"] - sf["x"]) ** 2)
        pow_x += np.sum(np.abs(sf["x"]) ** 2)
    db = lambda v: 10 * np.log10(v)
    assert abs(db(err_h / pow_h) - db(err_h_o / pow_h)) <= 0.1
    assert abs(db(err_x / pow_x) - db(err_x_o / pow_x)) <= 0.1


# ------------------------------------------------- differentiable receive (adjoint)
ADJ_CASES = [
    # M, K, N, n_fft, B, D
    (6, 2, 30, 64, 7, 3), (32, 4, 120, 256, 12, 6), (17, 5, 100, 256, 9, 4), (128, 16, 1200, 2048, 12, 6),
    (24, 3, 100, 256, 16, 3), (10, 2, 90, 256, 24, 2), (9, 2, 140, 256, 20, 2), (8, 3, 180, 256, 36, 3),
]


def _adj_inputs(M, K, N, nfft, B, D, seed):
    sh = synth.SubframeShape(M=M, K=K, n_sc=N, n_fft=nfft, n_taps=5 if nfft < 2048 else 24,
                             tau_rms=3.0 if nfft < 2048 else 6.0, snr_db=12.0, qam_bits=4, n_data_per_slot=D)
    sf = synth.make_subframe(sh, seed=seed)
    c64 = {k: synth.as_c64(sf[k]) for k in ("y_pilot", "pilots", "y_data", "x")}
    return sh, sf, c64


@pytest.mark.parametrize("case", ADJ_CASES)
def test_mse_backward_matches_the_differentiable_oracle(case):
    """Loss, dL/dW* (main and tail), the detector's dL/dsigma2 and the total gradient in
    (sigma2, tau) against torch.autograd of the FP64 oracle (FP32 adjoint: 1e-3 relative)."""
    M, K, N, nfft, B, D = case
    sh, sf, c64 = _adj_inputs(M, K, N, nfft, B, D, seed=synth.SEED_BASE + 50)
    s2, tau = 1.7 * sh.sigma2, 0.8 * sh.tau_rms          # off the generator's values
    p = params_for(sh, B)
    p.sigma2, p.tau_rms = s2, tau
    plan = R.Plan(p)
    s = plan.shapes()
    tail = plan.tail
    h = torch.empty(s["h"], dtype=torch.complex64, device="cuda")
    g_h = torch.empty_like(h)
    x = torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda")
    scal = torch.empty(2, dtype=torch.float32, device="cuda")
    gwm = torch.empty((B, B), dtype=torch.complex64, device="cuda")
    gwt = torch.empty((tail, tail), dtype=torch.complex64, device="cuda") if tail else None
    yp, pil, yd, xr = _dev(c64["y_pilot"]), _dev(c64["pilots"]), _dev(c64["y_data"]), _dev(c64["x"])
    R.rapro_receive_subframe(plan, yp, pil, yd, x, h_out=h)
    R.rapro_mse_backward(plan, yp, pil, yd, h, x, xr, g_h, scal, gwm, gwt)
    sc = _host(scal).astype(np.float64)
    kw = dict(B=B, n_taps=sh.n_taps, n_fft=sh.n_fft, n_data_per_slot=D, sigma2_est=s2, tau=tau, sigma2_det=s2)
    ins = [c64[k].astype(np.complex128) for k in ("y_pilot", "pilots", "y_data", "x")]
    loss_o, g_m, g_t, g_sd = G.weight_grads(*ins, **kw)
    assert abs(sc[0] - loss_o) <= 1e-5 * loss_o
    assert abs(sc[1] - g_sd) <= 1e-3 * abs(g_sd)
    assert np.linalg.norm(_host(gwm) - g_m) <= 1e-3 * np.linalg.norm(g_m)
    if tail:
        assert np.linalg.norm(_host(gwt) - g_t) <= 1e-3 * np.linalg.norm(g_t)
    _, g_se, g_tau, g_sd2 = G.grads(*ins, **kw)
    d_s2_w, d_tau = R.rapro_weight_grad_host(p, _host(gwm).astype(np.complex128),
                                             _host(gwt).astype(np.complex128) if tail else None)
    np.testing.assert_allclose([sc[1] + d_s2_w, d_tau], [g_se + g_sd2, g_tau], rtol=2e-3, atol=1e-9)


def test_autograd_function_and_adam_fit_of_the_channel_statistics():
    """torch.autograd.Function over the CUDA forward and adjoint: its gradient matches central
    differences of the CUDA loss, and 200 Adam steps from (2 sigma2, 2 tau) lower the loss to
    that at the true statistics and move (sigma2, tau) towards them."""
    from paper_1802_05427_gb300 import autograd as AG
    sh = synth.SubframeShape(M=64, K=8, n_sc=600, n_fft=1024, n_taps=16, tau_rms=6.0, snr_db=15.0,
                             qam_bits=4)
    B = 12
    batch = []
    for i in range(4):
        sf = synth.make_subframe(sh, seed=synth.SEED_BASE + 60 + i)
        batch.append({k: _dev(synth.as_c64(sf[k])) for k in ("y_pilot", "pilots", "y_data")})
        batch[-1]["x_ref"] = _dev(synth.as_c64(sf["x"]))
    shape = dict(M=sh.M, K=sh.K, n_sc=sh.n_sc, n_fft=sh.n_fft, subblock=B, qam_bits=sh.qam_bits, n_taps=sh.n_taps)
    theta = torch.tensor([2 * sh.sigma2, 2 * sh.tau_rms], dtype=torch.float64, requires_grad=True)
    loss = AG.symbol_mse(theta, batch, shape)
    loss.backward()
    for i, rel in ((0, 1e-2), (1, 1e-2)):
        e = torch.zeros(2, dtype=torch.float64)
        step = 1e-2 * float(theta.detach()[i])
        e[i] = step
        fd = (float(AG.symbol_mse(theta.detach() + e, batch, shape)) -
              float(AG.symbol_mse(theta.detach() - e, batch, shape))) / (2 * step)
        assert abs(float(theta.grad[i]) - fd) <= rel * abs(fd) + 1e-7, (i, float(theta.grad[i]), fd)
    truth = torch.tensor([sh.sigma2, sh.tau_rms], dtype=torch.float64)
    l_true = float(AG.symbol_mse(truth, batch, shape))
    log_theta = torch.log(theta.detach()).clone().requires_grad_(True)
    opt = torch.optim.Adam([log_theta], lr=0.05)
    l0 = None
    for it in range(200):
        opt.zero_grad()
        l = AG.symbol_mse(torch.exp(log_theta), batch, shape)
        if l0 is None:
            l0 = float(l.detach())
        l.backward()
        opt.step()
    fit = torch.exp(log_theta.detach())
    l_fit = float(AG.symbol_mse(fit, batch, shape))
    assert l_fit < l0 and l_fit <= 1.01 * l_true, (l0, l_fit, l_true)
    for i in range(2):
        assert abs(np.log(float(fit[i] / truth[i]))) < 0.5 * np.log(2.0), (fit, truth)


# ----------------------------------------------- batched heterogeneous receive + tuner
BATCH_JOBS = [
    # shape, B, layout ("orth" | "comb"), precision
    (synth.SubframeShape(M=32, K=4, n_sc=72, n_fft=128, snr_db=12.0, qam_bits=2), 12, "orth", R.RAPRO_PREC_FP32),
    (synth.SubframeShape(M=64, K=8, n_sc=300, n_fft=512, snr_db=18.0, qam_bits=4), 48, "orth", R.RAPRO_PREC_FP32),
    (synth.SubframeShape(M=128, K=12, n_sc=600, n_fft=1024, snr_db=20.0, qam_bits=6), 12, "orth", R.RAPRO_PREC_FP32),
    (synth.SubframeShape(M=20, K=16, n_sc=96, n_fft=128, snr_db=25.0, qam_bits=4), 16, "orth", R.RAPRO_PREC_BF16),
    (synth.SubframeShape(M=40, K=6, n_sc=144, n_fft=256, snr_db=15.0, qam_bits=2), 0, "comb", R.RAPRO_PREC_FP32),
    (synth.SubframeShape(M=13, K=3, n_sc=75, n_fft=128, snr_db=10.0, qam_bits=2), 10, "orth", R.RAPRO_PREC_FP32),
]


def _batch_job(i, sh, B, layout, prec):
    if layout == "comb":
        sf = synth.make_comb_subframe(sh, seed=synth.SEED_BASE + 70 + i, S=12)
        p = comb_params(sh, 12, R.RAPRO_COMB_SW)
    else:
        sf = synth.make_subframe(sh, seed=synth.SEED_BASE + 70 + i)
        p = params_for(sh, B)
        p.precision = prec
    c64 = {k: synth.as_c64(sf[k]) for k in ("y_pilot", "pilots", "y_data")}
    plan = R.Plan(p)
    s = plan.shapes()
    job = dict(plan=plan, y_pilot=_dev(c64["y_pilot"]), pilots=_dev(c64["pilots"]), y_data=_dev(c64["y_data"]),
               x_eq=torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda"),
               labels=torch.empty(s["labels"], dtype=torch.uint8, device="cuda"),
               llr=torch.empty(s["llr"], dtype=torch.float32, device="cuda"),
               info=torch.full(s["info"], -7, dtype=torch.int32, device="cuda"),
               h_out=torch.empty(s["h"], dtype=torch.complex64, device="cuda"))
    if layout == "comb":
        o = O.comb_receive_subframe(c64["y_pilot"].astype(np.complex128), c64["pilots"].astype(np.complex128),
                                    c64["y_data"].astype(np.complex128), K=sh.K, S=12, method=O.COMB_SW,
                                    sigma2=sh.sigma2, r=oracle_r(sh), n_data_per_slot=sh.n_data_per_slot,
                                    q=sh.qam_bits)
    else:
        o = oracle_receive(sh, c64, B)
    return job, o


def _check_job(job, o, sh, prec):
    h_tol = TOL_BF16 if prec == R.RAPRO_PREC_BF16 else TOL
    assert_parity(_host(job["h_out"]), o["h"], (2, 3), h_tol)
    assert (_host(job["info"]) == 0).all()
    if prec == R.RAPRO_PREC_FP32:
        check_detection(dict(x_eq=_host(job["x_eq"]), labels=_host(job["labels"]), llr=_host(job["llr"])), o,
                        sh.qam_bits)


def test_receive_batch_of_uneven_jobs_matches_the_oracle_eager_and_in_a_graph():
    jobs, refs = [], []
    for i, (sh, B, layout, prec) in enumerate(BATCH_JOBS):
        j, o = _batch_job(i, sh, B, layout, prec)
        jobs.append(j)
        refs.append(o)
    batch = R.Batch(4)
    R.rapro_receive_batch(batch, jobs)
    torch.cuda.synchronize()
    for j, o, (sh, B, layout, prec) in zip(jobs, refs, BATCH_JOBS):
        _check_job(j, o, sh, prec)
    first = [_host(j["x_eq"]).copy() for j in jobs]
    for j in jobs:
        j["x_eq"].zero_()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            R.rapro_receive_batch(batch, jobs, stream=st)
    g.replay()
    torch.cuda.synchronize()
    for j, x0 in zip(jobs, first):
        np.testing.assert_array_equal(_host(j["x_eq"]), x0)
    for j in jobs:
        assert j["plan"].device_status() == 0
    shared = dict(jobs[0])
    shared["h_out"] = None
    with pytest.raises(R.RaproError):
        R.rapro_receive_batch(batch, [shared, dict(shared)])
    batch.close()


@pytest.mark.parametrize("case", [(8, 2, 72, 128, 12), (128, 12, 1200, 2048, 12), (64, 8, 300, 512, 48),
                                  (20, 5, 100, 256, 10)])
def test_autotuner_picks_an_applicable_kernel_and_keeps_parity(case):
    M, K, N, nfft, B = case
    sh = synth.SubframeShape(M=M, K=K, n_sc=N, n_fft=nfft, n_taps=24 if nfft >= 2048 else 6,
                             tau_rms=8.0 if nfft >= 2048 else 4.0, snr_db=12.0, qam_bits=4)
    sf, c64 = _inputs(sh, 9)
    plan = R.Plan(params_for(sh, B))
    s = plan.shapes()
    yp, pil, yd = _dev(c64["y_pilot"]), _dev(c64["pilots"]), _dev(c64["y_data"])
    h = torch.empty(s["h"], dtype=torch.complex64, device="cuda")
    x = torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda")
    assert R.rapro_plan_variant(plan)[0] == -1
    R.rapro_plan_tune(plan, yp, pil, yd, h, x)
    ev, split, grid = R.rapro_plan_variant(plan)
    assert ev in (0, 1, 2, 3, 4) and split in (1, 2) and grid in (0, 1)
    if B > 32:
        assert ev in (3, 4)                 # tiled FP32 or the tensor-core GEMM
    if B > 16:
        assert not R.rapro_receive_is_fused(plan, yp, yd)   # the fused form does not apply
    lab = torch.empty(s["labels"], dtype=torch.uint8, device="cuda")
    llr = torch.empty(s["llr"], dtype=torch.float32, device="cuda")
    R.rapro_receive_subframe(plan, yp, pil, yd, x, lab, llr, h_out=h)
    o = oracle_receive(sh, c64, B)
    assert_parity(_host(h), o["h"], (2, 3), TOL)
    check_detection(dict(x_eq=_host(x), labels=_host(lab), llr=_host(llr)), o, sh.qam_bits)


@pytest.mark.parametrize("case", [(20, 12, 96, 128, 12), (16, 5, 100, 256, 10)])
def test_every_kernel_choice_keeps_parity(case):
    """Each estimator kernel that applies, one or two detector warps per role and one or as
    many estimator CTAs per SM as fit: the same results as the oracle."""
    M, K, N, nfft, B = case
    sh = synth.SubframeShape(M=M, K=K, n_sc=N, n_fft=nfft, snr_db=14.0, qam_bits=4)
    sf, c64 = _inputs(sh, 21)
    o = oracle_receive(sh, c64, B)
    plan = R.Plan(params_for(sh, B))
    s = plan.shapes()
    assert R.rapro_plan_variant(plan) == (-1, 1, 1)                  # the throughput defaults
    yp, pil, yd = _dev(c64["y_pilot"]), _dev(c64["pilots"]), _dev(c64["y_data"])
    for ev in (-1, 0, 1, 2, 3, 4):
        for split in (1, 2):
            for grid in (0, 1):
                R.rapro_plan_set_variant(plan, ev, split, grid)
                assert R.rapro_plan_variant(plan) == (ev, split, grid)
                h = torch.empty(s["h"], dtype=torch.complex64, device="cuda")
                x = torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda")
                lab = torch.empty(s["labels"], dtype=torch.uint8, device="cuda")
                llr = torch.empty(s["llr"], dtype=torch.float32, device="cuda")
                R.rapro_receive_subframe(plan, yp, pil, yd, x, lab, llr, h_out=h)
                assert_parity(_host(h), o["h"], (2, 3), TOL, what=str((ev, split, grid)))
                check_detection(dict(x_eq=_host(x), labels=_host(lab), llr=_host(llr)), o, sh.qam_bits)
    for bad in ((5, 1, 1), (-2, 1, 1), (-1, 0, 1), (-1, 3, 1), (-1, 1, 9), (-1, 1, -1)):
        with pytest.raises(R.RaproError):
            R.rapro_plan_set_variant(plan, *bad)
    assert R.rapro_plan_variant(plan) == (4, 2, 1)                   # a bad call changes nothing
    assert plan.device_status() == 0
    plan.close()


def test_bf16_form_falls_back_to_fp64_on_ill_conditioned_subcarriers():
    """Users 0 and 1 nearly collinear on two subcarriers with a tiny sigma2: cond(A) ~ 1e8.
    The precision form re-solves those subcarriers in FP64 (agreeing with the FP64 oracle),
    where the FP32 detector alone is far off."""
    sh = synth.SubframeShape(M=16, K=4, n_sc=32, n_fft=64, snr_db=90.0, qam_bits=2)
    sf, c64 = _inputs(sh, 12)
    rng = np.random.default_rng(1)
    h = np.broadcast_to(np.transpose(sf["H"], (1, 0, 2))[None], (sh.n_slots, sh.K, sh.M, sh.n_sc)).copy()
    bad = [3, 17]
    for n in bad:
        h[:, 1, :, n] = h[:, 0, :, n] + 1e-4 * (rng.standard_normal((sh.n_slots, sh.M)) +
                                                1j * rng.standard_normal((sh.n_slots, sh.M)))
    h = synth.as_c64(h)
    x_o, _ = O.mmse_detect(h.astype(np.complex128), c64["y_data"].astype(np.complex128), sh.sigma2,
                           sh.n_data_per_slot)
    out = {}
    for prec in (R.RAPRO_PREC_BF16, R.RAPRO_PREC_FP16, R.RAPRO_PREC_FP32):
        p = params_for(sh, 8)
        p.precision = prec
        plan = R.Plan(p)
        s = plan.shapes()
        x = torch.empty(s["x_eq"], dtype=torch.complex64, device="cuda")
        info = torch.full(s["info"], -7, dtype=torch.int32, device="cuda")
        R.rapro_mmse_detect(plan, _dev(h), _dev(c64["y_data"]), x, info=info)
        out[prec] = (_host(x), _host(info))
    good = np.setdiff1d(np.arange(sh.n_sc), bad)
    for prec in (R.RAPRO_PREC_BF16, R.RAPRO_PREC_FP16):
        x_b, info_b = out[prec]
        assert (info_b == 0).all()
        # per subcarrier: the FP64 re-solves of the flagged ones at the FP32 bar, the rest at
        # the 16-bit filter's effect on a well-conditioned solve
        assert_parity(x_b[..., bad], x_o[..., bad], (0, 1), 1e-5, what="fp64 fallback")
        assert_parity(x_b[..., good], x_o[..., good], (0, 1), 1e-4, what="well-conditioned")
    x_f, _ = out[R.RAPRO_PREC_FP32]
    assert rel_err_per(x_f, x_o, axes=(0, 1))[bad].min() > 1e-3 or not np.isfinite(x_f[..., bad]).all()


def test_receiver_pipelines_host_subframes_correctly():
    """Receiver.receive_host with two buffer sets in flight: every subframe's results match
    the oracle (the overlap of copies and kernels changes no result)."""
    sh = synth.SubframeShape(M=32, K=4, n_sc=120, n_fft=256, snr_db=15.0, qam_bits=4)
    rx = R.Receiver(params_for(sh, 12), depth=2)
    s = rx.plan.shapes()
    subframes, outs = [], []
    for i in range(4):
        sf, c64 = _inputs(sh, synth.SEED_BASE + 80 + i)
        subframes.append(c64)
        host = {k: torch.from_numpy(c64[k]).pin_memory() for k in ("y_pilot", "pilots", "y_data")}
        x_h = torch.empty(s["x_eq"], dtype=torch.complex64).pin_memory()
        lab_h = torch.empty(s["labels"], dtype=torch.uint8).pin_memory()
        outs.append((host, x_h, lab_h))
    rx.fork()
    for host, x_h, lab_h in outs:
        rx.receive_host(host["y_pilot"], host["pilots"], host["y_data"], x_h, lab_h)
    rx.join()
    torch.cuda.synchronize()
    for c64, (_, x_h, lab_h) in zip(subframes, outs):
        o = oracle_receive(sh, c64, 12)
        assert_parity(x_h.numpy(), o["x_eq"], (2,), TOL)
        margin = O.boundary_margin(o["xhat"], sh.qam_bits)
        far = margin > MARGIN
        assert (lab_h.numpy()[far] == o["labels"][far]).all()


def test_new_entry_points_reject_bad_arguments():
    """Argument checks of the comb, adjoint, tuner and batch entry points (no launch)."""
    sh = synth.TINY
    orth = R.Plan(params_for(sh, 12))
    comb = R.Plan(comb_params(sh, 6, R.RAPRO_COMB_3W))
    so, sc = orth.shapes(), comb.shapes()
    z = lambda shape, dt=torch.complex64: torch.zeros(shape, dtype=dt, device="cuda")
    # the adjoint reads the orthogonal layout
    with pytest.raises(R.RaproError) as e:
        R.rapro_mse_backward(comb, z(sc["y_pilot"]), z(sc["pilots"]), z(sc["y_data"]), z(sc["h"]), z(sc["x_eq"]),
                             z(sc["x_eq"]), z(sc["h"]), z((2,), torch.float32), z((0, 0)))
    assert e.value.status in (R.RAPRO_ERR_UNSUPPORTED, R.RAPRO_ERR_INVALID_ARG)
    # the adjoint supports B <= 64
    big = R.Plan(params_for(synth.SubframeShape(M=4, K=2, n_sc=72, n_fft=128), 72))
    sb = big.shapes()
    with pytest.raises(R.RaproError) as e:
        R.rapro_mse_backward(big, z(sb["y_pilot"]), z(sb["pilots"]), z(sb["y_data"]), z(sb["h"]), z(sb["x_eq"]),
                             z(sb["x_eq"]), z(sb["h"]), z((2,), torch.float32), z((72, 72)))
    assert e.value.status == R.RAPRO_ERR_UNSUPPORTED
    # g_h must not alias an input
    h = z(so["h"])
    with pytest.raises(R.RaproError) as e:
        R.rapro_mse_backward(orth, z(so["y_pilot"]), z(so["pilots"]), z(so["y_data"]), h, z(so["x_eq"]),
                             z(so["x_eq"]), h, z((2,), torch.float32), z((12, 12)))
    assert e.value.status == R.RAPRO_ERR_INVALID_ARG
    # the weight gradient covers the exponential model only
    pu = params_for(sh, 12, pdp="uniform_L")
    with pytest.raises(R.RaproError):
        R.rapro_weight_grad_host(pu, np.zeros((12, 12), np.complex128))
    # batch: a pool of 0 or 33 streams, a job without arrays
    for n in (0, 33):
        with pytest.raises(R.RaproError):
            R.Batch(n)
    b = R.Batch(2)
    arr = (R.RaproJob * 1)()
    arr[0].plan = orth.handle.value
    with pytest.raises(R.RaproError):
        R._check(R.lib().rapro_receive_batch(b.handle, arr, 1, None), "rapro_receive_batch")
    assert R.lib().rapro_receive_batch(b.handle, None, 0, None) == R.RAPRO_OK
    b.close()
    # the tuner needs every array
    assert R.lib().rapro_plan_tune(orth.handle, None, None, None, None, None, None) == R.RAPRO_ERR_INVALID_ARG


def test_detector_wait_that_runs_out_reports_a_timeout_and_writes_nothing():
    """Timeout path of the pipeline waits, made to happen without a fault: the diagnostic
    setting gives the detector's producer/consumer waits a short limit and stops its load
    producer, so the consumers' first wait runs out.  The kernel records RAPRO_ERR_TIMEOUT
    in the plan's status word, writes no output or info entry and returns; the context stays
    usable, and with the setting off the next call matches the oracle."""
    import time
    sh = synth.SubframeShape(M=32, K=4, n_sc=64, n_fft=128, snr_db=15.0, qam_bits=4)
    sf, c64 = _inputs(sh, 51)
    h_ls = O.ls_estimate(c64["y_pilot"].astype(np.complex128), c64["pilots"].astype(np.complex128))
    h = synth.as_c64(O.subblock_lmmse(h_ls, 8, oracle_r(sh), sh.sigma2))
    plan = R.Plan(params_for(sh, 8))
    s = plan.shapes()
    hd, yd = _dev(h), _dev(c64["y_data"])
    x = torch.full(s["x_eq"], float("nan"), dtype=torch.complex64, device="cuda")
    lab = torch.full(s["labels"], 7, dtype=torch.uint8, device="cuda")
    info = torch.full(s["info"], -7, dtype=torch.int32, device="cuda")
    R.rapro_plan_set_wait_test(plan, True, 64)          # <= 64 rounds of <= 2 us per wait
    torch.cuda.synchronize()
    t0 = time.time()
    R.rapro_mmse_detect(plan, hd, yd, x, lab, None, info)
    torch.cuda.synchronize()
    assert time.time() - t0 < 1.0                       # returned after the short limit
    assert plan.device_status(reset=True) == R.RAPRO_ERR_TIMEOUT
    assert np.isnan(_host(x)).all() and (_host(lab) == 7).all() and (_host(info) == -7).all()
    R.rapro_plan_set_wait_test(plan, False, 0)
    R.rapro_mmse_detect(plan, hd, yd, x, lab, None, info)
    assert plan.device_status() == 0
    x_o, _ = O.mmse_detect(h.astype(np.complex128), c64["y_data"].astype(np.complex128), sh.sigma2,
                           sh.n_data_per_slot)
    assert_parity(_host(x), x_o, (2,), TOL, what="after the timeout")
    assert (_host(info) == 0).all()
    plan.close()


def test_autograd_with_learnable_block_weights_matches_the_oracle():
    """The block weights of Eq. 12 as autograd parameters (tied over the full blocks, the tail's
    own) with the detector's sigma2: loss, torch gradients of W_main, W_tail and sigma2 against
    torch.autograd of the FP64 oracle given the same weights (FP32 adjoint: 1e-3 relative),
    and a few Adam steps on W that lower the loss."""
    from paper_1802_05427_gb300 import autograd as AG
    M, K, N, nfft, B, D = 16, 4, 100, 256, 12, 3
    sh, sf, c64 = _adj_inputs(M, K, N, nfft, B, D, seed=synth.SEED_BASE + 57)
    tail = N % B
    rng = np.random.default_rng(5)
    s_e, ta = torch.tensor(sh.sigma2, dtype=torch.float64), torch.tensor(sh.tau_rms, dtype=torch.float64)
    pert = lambda n: 0.05 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    wm0 = (G.block_weight(B, s_e, ta, sh.n_taps, sh.n_fft).numpy() + pert(B)).astype(np.complex64)
    wt0 = (G.block_weight(tail, s_e, ta, sh.n_taps, sh.n_fft).numpy() + pert(tail)).astype(np.complex64)
    s2_0 = 1.5 * sh.sigma2
    batch = [dict(y_pilot=_dev(c64["y_pilot"]), pilots=_dev(c64["pilots"]), y_data=_dev(c64["y_data"]),
                  x_ref=_dev(c64["x"]))]
    shape = dict(M=M, K=K, n_sc=N, n_fft=nfft, subblock=B, qam_bits=sh.qam_bits, n_taps=sh.n_taps,
                 tau_rms=sh.tau_rms, n_sym=2 * (D + 1), n_pilot_sym=2)
    wm = torch.tensor(wm0, dtype=torch.complex128, requires_grad=True)
    wt = torch.tensor(wt0, dtype=torch.complex128, requires_grad=True)
    s2 = torch.tensor(s2_0, dtype=torch.float64, requires_grad=True)
    loss = AG.symbol_mse_weights(wm, wt, s2, batch, shape)
    loss.backward()
    wm_o = torch.tensor(wm0, dtype=torch.complex128, requires_grad=True)
    wt_o = torch.tensor(wt0, dtype=torch.complex128, requires_grad=True)
    s2_o = torch.tensor(s2_0, dtype=torch.float64, requires_grad=True)
    ins = [c64[k].astype(np.complex128) for k in ("y_pilot", "pilots", "y_data", "x")]
    loss_o, _ = G.symbol_mse(*ins, B=B, n_taps=sh.n_taps, n_fft=nfft, n_data_per_slot=D, sigma2_est=s_e, tau=ta,
                             sigma2_det=s2_o, weights=(wm_o, wt_o))
    loss_o.backward()
    assert abs(float(loss) - float(loss_o)) <= 1e-5 * float(loss_o)
    for g, go in ((wm.grad, wm_o.grad), (wt.grad, wt_o.grad)):
        assert torch.linalg.norm(g - go) <= 1e-3 * torch.linalg.norm(go)
    assert abs(float(s2.grad) - float(s2_o.grad)) <= 1e-3 * abs(float(s2_o.grad))
    # learning the weights from the pilots and known symbols lowers the loss
    opt = torch.optim.Adam([wm, wt], lr=2e-3)
    l0 = float(loss)
    for _ in range(20):
        opt.zero_grad()
        l = AG.symbol_mse_weights(wm, wt, s2.detach(), batch, shape)
        l.backward()
        opt.step()
    assert float(AG.symbol_mse_weights(wm, wt, s2.detach(), batch, shape)) < l0
