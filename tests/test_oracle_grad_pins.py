"""Pins of the differentiable oracle: its autograd gradients against central finite
differences of the independent numpy oracle's forward pass (FP64, h = 1e-4)."""
import numpy as np
import pytest

from oracle import rapro_oracle as O
from oracle import rapro_grad_oracle as G
from paper_1802_05427_gb300 import synth


def _case(seed=3, **kw):
    base = dict(M=6, K=2, n_sc=30, n_fft=64, n_taps=5, tau_rms=3.0, snr_db=12.0, qam_bits=2, n_data_per_slot=3)
    base.update(kw)
    sh = synth.SubframeShape(**base)
    sf = synth.make_subframe(sh, seed=seed)
    return sh, sf


def _np_loss(sh, sf, B, s_est, tau, s_det, weights=None):
    """The numpy oracle's forward: Eq. 9 -> Eq. 12/17 -> Eq. 22, then mean |x~ - x|^2."""
    r = O.make_r("exp", n_taps=sh.n_taps, tau_rms=tau, n_fft=sh.n_fft)
    h_ls = O.ls_estimate(sf["y_pilot"], sf["pilots"])
    h = O.subblock_lmmse(h_ls, B, r, s_est, weights=weights)
    x_eq, _ = O.mmse_detect(h, sf["y_data"], s_det, sh.n_data_per_slot)
    return float(np.mean(np.abs(x_eq - sf["x"]) ** 2))


@pytest.mark.parametrize("B", [5, 7, 30])
def test_autograd_gradients_match_central_differences(B):
    sh, sf = _case()
    s_est, tau, s_det = 0.09, 2.2, 0.05          # off the generator's values, as in a fit
    loss, g_se, g_tau, g_sd = G.grads(sf["y_pilot"], sf["pilots"], sf["y_data"], sf["x"], B=B,
                                      n_taps=sh.n_taps, n_fft=sh.n_fft, n_data_per_slot=sh.n_data_per_slot,
                                      sigma2_est=s_est, tau=tau, sigma2_det=s_det)
    assert abs(loss - _np_loss(sh, sf, B, s_est, tau, s_det)) < 1e-12 * max(1.0, loss)
    h = 1e-4
    fd = lambda f, v: (f(v * (1 + h)) - f(v * (1 - h))) / (2 * h * v)
    fd_se = fd(lambda v: _np_loss(sh, sf, B, v, tau, s_det), s_est)
    fd_tau = fd(lambda v: _np_loss(sh, sf, B, s_est, v, s_det), tau)
    fd_sd = fd(lambda v: _np_loss(sh, sf, B, s_est, tau, v), s_det)
    for g, f in ((g_se, fd_se), (g_tau, fd_tau), (g_sd, fd_sd)):
        assert abs(g - f) <= 1e-6 * max(abs(f), 1e-3), (g, f)


def test_weight_gradient_matches_central_differences():
    """G = dL/dW* with dL = 2 Re sum conj(G) dW: dL/dRe W = 2 Re G, dL/dIm W = 2 Im G."""
    sh, sf = _case(seed=4)
    B, s_est, tau, s_det = 12, 0.07, 2.5, 0.06
    loss, g_m, g_t, g_sd = G.weight_grads(sf["y_pilot"], sf["pilots"], sf["y_data"], sf["x"], B=B,
                                          n_taps=sh.n_taps, n_fft=sh.n_fft, n_data_per_slot=sh.n_data_per_slot,
                                          sigma2_est=s_est, tau=tau, sigma2_det=s_det)
    r = O.make_r("exp", n_taps=sh.n_taps, tau_rms=tau, n_fft=sh.n_fft)
    base = O.subblock_weights(sh.n_sc, B, r, s_est)
    rng = np.random.default_rng(0)
    h = 1e-5
    for which, g in (("main", g_m), ("tail", g_t)):
        for _ in range(4):
            i, j = rng.integers(0, g.shape[0], size=2)
            for unit, part in ((1.0, np.real), (1j, np.imag)):
                def f(eps):
                    ws = []
                    for b0, W in base:
                        W = W.copy()
                        if (W.shape[0] == B) == (which == "main"):
                            W[i, j] += eps * unit
                        ws.append((b0, W))
                    return _np_loss(sh, sf, B, s_est, tau, s_det, weights=ws)
                fd = (f(h) - f(-h)) / (2 * h)
                assert abs(2 * part(g[i, j]) - fd) <= 1e-6 * max(abs(fd), 1e-4), (which, i, j, g[i, j], fd)
