"""CPU tests of the C-ABI library: it builds, loads, exports what rapro.h declares, and its
host-side logic (parameter checks, FP64 weights) behaves.  No GPU calls."""
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
    ("pilot_layout", R.RAPRO_PILOT_COMB, R.RAPRO_ERR_UNSUPPORTED),
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
