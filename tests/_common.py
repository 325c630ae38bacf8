"""Shared test helpers: workload shapes, parameter sets, oracle runs, comparisons."""
import numpy as np

from paper_1802_05427_gb300 import synth


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
