"""Shared test helpers: workload shapes, parameter sets, oracle runs, comparisons."""
import numpy as np

from paper_1802_05427_gb300 import synth

# Element-wise bar, in units of the norm-wise tolerance times the rms of the reference over
# the same group.  Rounding errors of the device arithmetic are small, nearly independent
# per element and of similar size across a group, so the largest of n of them sits about
# sqrt(2 ln n) rms errors out (~5 for the 153,600 entries of one (slot, user) slice of h at
# 128 x 1200, ~4 for 1,200 subcarriers of x~).  A group that meets the norm-wise bar then
# has max |a - b| <= ~5 tol rms(b); 30 leaves headroom for heavier tails (ill-conditioned
# subcarriers, where the K x K solve amplifies the error) while a single wrong element, a
# tile-edge column or a misplaced box, off by O(rms(b)), is caught by a factor of ~3000.
ELEM_C = 30.0


def params_for(sh: synth.SubframeShape, B: int, pdp: str = "exp", L: float = 8.0):
    from paper_1802_05427_gb300 import rapro as R
    return R.make_params(M=sh.M, K=sh.K, n_sc=sh.n_sc, n_fft=sh.n_fft, subblock=B, sigma2=sh.sigma2,
                         qam_bits=sh.qam_bits, n_sym=sh.n_slots * (sh.n_data_per_slot + 1),
                         n_pilot_sym=sh.n_slots,
                         pdp=R.RAPRO_PDP_EXP if pdp == "exp" else R.RAPRO_PDP_UNIFORM_L,
                         n_taps=sh.n_taps, tau_rms=sh.tau_rms, L=L)


def oracle_r(sh: synth.SubframeShape, pdp: str = "exp", L: float = 8.0):
    from oracle import rapro_oracle as O
    if pdp == "exp":
        return O.make_r("exp", n_taps=sh.n_taps, tau_rms=sh.tau_rms, n_fft=sh.n_fft)
    return O.make_r("uniform_L", L=L, n=sh.n_fft)


def rel_err_per(a, b, axes):
    """Norm-wise relative error ||a - b|| / ||b|| over ``axes`` (one value per remaining index)."""
    num = np.sqrt(np.sum(np.abs(np.asarray(a, np.complex128) - b) ** 2, axis=axes))
    den = np.sqrt(np.sum(np.abs(b) ** 2, axis=axes))
    return num / np.maximum(den, 1e-300)


def elem_err_per(a, b, axes):
    """max |a - b| / rms(b) over ``axes`` (one value per remaining index)."""
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    d = np.abs(a - b)
    n = np.prod([b.shape[ax] for ax in axes])
    rms = np.sqrt(np.sum(np.abs(b) ** 2, axis=axes) / max(n, 1))
    return np.max(d, axis=axes) / np.maximum(rms, 1e-300)


def assert_parity(a, b, axes, tol, what="", c=ELEM_C):
    """Both bars per group over ``axes``: ||a - b|| / ||b|| <= tol, and every element
    max |a - b| <= c tol rms(b).  Returns the worst (norm-wise, element-wise / rms) errors."""
    e_n = rel_err_per(a, b, axes)
    e_e = elem_err_per(a, b, axes)
    assert e_n.max() <= tol, f"{what} norm-wise rel err {e_n.max():.3g} > {tol:g}"
    assert e_e.max() <= c * tol, f"{what} element err {e_e.max():.3g} rms > {c:g} x {tol:g}"
    return float(e_n.max()), float(e_e.max())
