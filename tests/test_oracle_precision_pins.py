"""Pins of the oracle's precision-form pieces (CPU): the two sides of Eq. 22, the 16-bit
rounding model of tensor-core operands, and one step of iterative refinement."""
import numpy as np
import pytest

from oracle import rapro_oracle as O


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_gram_and_matched_filter_against_an_antenna_by_antenna_sum():
    rng = np.random.default_rng(3)
    T, K, M, N, D = 2, 3, 5, 4, 2
    h, y = _rand(rng, (T, K, M, N)), _rand(rng, (T * D, M, N))
    A, z = O.gram_matched_filter(h, y, 0.25, D)
    for t in range(T):
        for k in range(N):
            Ab = 0.25 * np.eye(K, dtype=complex)
            zb = np.zeros((K, D), dtype=complex)
            for m in range(M):                    # rank-one updates, one antenna at a time
                hm = h[t, :, m, k]
                Ab += np.outer(np.conj(hm), hm)
                zb += np.outer(np.conj(hm), y[t * D:(t + 1) * D, m, k])
            np.testing.assert_allclose(A[t, k], Ab, rtol=1e-13, atol=1e-13)
            np.testing.assert_allclose(z[t, k], zb, rtol=1e-13, atol=1e-13)
            assert np.allclose(A[t, k], np.conj(A[t, k].T))
            assert np.linalg.eigvalsh(A[t, k]).min() >= 0.25 - 1e-12


def test_gram_solves_to_the_mmse_output():
    """A^-1 z is the detector output of Eq. 22 computed by mmse_detect."""
    rng = np.random.default_rng(4)
    T, K, M, N, D = 2, 4, 16, 6, 3
    h, y = _rand(rng, (T, K, M, N)), _rand(rng, (T * D, M, N))
    A, z = O.gram_matched_filter(h, y, 0.1, D)
    x, _ = O.mmse_detect(h, y, 0.1, D)
    for t in range(T):
        xs = np.linalg.solve(A[t], z[t])                 # [N][K][D]
        np.testing.assert_allclose(np.transpose(xs, (2, 1, 0)), x[t * D:(t + 1) * D], rtol=1e-11, atol=1e-12)


def _bf16_neighbours(v):
    """The two BF16 values around the float32 v (brute force over the bit pattern)."""
    u = np.float32(v).view(np.uint32)
    lo = np.uint32(u & np.uint32(0xFFFF0000)).view(np.float32)
    hi = np.uint32((u & np.uint32(0xFFFF0000)) + np.uint32(0x10000)).view(np.float32)
    return float(lo), float(hi)


def test_bf16_rounding_is_nearest_with_ties_to_even():
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-20, 20, 2000),
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0]]).astype(np.float32)
    r = O.round_half(x.astype(np.float64), "bf16")
    for v, got in zip(x, r):
        lo, hi = _bf16_neighbours(v)
        cands = sorted({lo, hi}, key=lambda c: (abs(c - float(v)),
                                                int(np.float32(c).view(np.uint32) >> 16) & 1))
        assert got == cands[0], (v, got, cands)
    assert O.round_half(np.array([1.0 + 2.0 ** -8]), "bf16")[0] == 1.0            # tie: even
    assert O.round_half(np.array([1.0 + 3 * 2.0 ** -8]), "bf16")[0] == 1.0 + 2.0 ** -6


def test_fp16_rounding_matches_ieee_binary16():
    x = np.array([1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 65504.0, 1e-8, -3.3333])
    np.testing.assert_array_equal(O.round_half(x, "fp16"), x.astype(np.float16).astype(np.float64))
    assert O.round_half(np.array([1.0 + 2.0 ** -11]), "fp16")[0] == 1.0


def test_refinement_with_the_exact_system_changes_nothing():
    rng = np.random.default_rng(6)
    T, K, M, N, D = 2, 3, 12, 5, 2
    h, y = _rand(rng, (T, K, M, N)), _rand(rng, (T * D, M, N))
    A, z = O.gram_matched_filter(h, y, 0.2, D)
    x1, s1 = O.refined_mmse_detect(h, y, 0.2, D, A, z)
    x, s = O.mmse_detect(h, y, 0.2, D)
    np.testing.assert_allclose(x1, x, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(s1, s, rtol=1e-12)


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_one_refinement_step_contracts_the_error(fmt):
    """With the system built from 16-bit-rounded H and y, x0 is off by about cond(A) x the
    rounding; one step brings it down by the factor ||A_low^-1 (A_low - A)|| (the classic
    bound of iterative refinement), checked per subcarrier."""
    rng = np.random.default_rng(7)
    T, K, M, N, D = 1, 6, 64, 16, 4
    h, y = _rand(rng, (T, K, M, N)) / np.sqrt(2), _rand(rng, (T * D, M, N)) / np.sqrt(2)
    sigma2 = 0.05
    A_low, z_low = O.gram_matched_filter(O.round_half(h, fmt), O.round_half(y, fmt), sigma2, D)
    A, _ = O.gram_matched_filter(h, y, sigma2, D)
    x, _ = O.mmse_detect(h, y, sigma2, D)
    x1, _ = O.refined_mmse_detect(h, y, sigma2, D, A_low, z_low)
    for k in range(N):
        x0 = np.linalg.solve(A_low[0, k], z_low[0, k])             # [K][D]
        xe = x[:, :, k].T
        e0 = np.linalg.norm(x0 - xe)
        e1 = np.linalg.norm(x1[:, :, k].T - xe)
        rho = np.linalg.norm(np.linalg.solve(A_low[0, k], A_low[0, k] - A[0, k]), 2)
        assert rho < 0.1
        assert e1 <= rho * e0 * (1 + 1e-6) + 1e-12, (k, e1, rho, e0)
        assert e1 < 0.1 * e0


def test_refinement_k1_closed_form():
    """K = 1: x1 = x0 + (z - a x0) / a_low with a = |h|^2 + sigma2, z = h^H y (scalars)."""
    rng = np.random.default_rng(8)
    h, y = _rand(rng, (1, 1, 7, 3)), _rand(rng, (2, 7, 3))
    A_low = np.full((1, 3, 1, 1), 5.0 + 0j)
    z_low = np.full((1, 3, 1, 2), 1.0 + 1.0j)
    x1, s = O.refined_mmse_detect(h, y, 0.3, 2, A_low, z_low)
    for k in range(3):
        hk = h[0, 0, :, k]
        a = np.vdot(hk, hk).real + 0.3
        for n in range(2):
            z = np.vdot(hk, y[n, :, k])
            x0 = (1.0 + 1.0j) / 5.0
            assert np.isclose(x1[n, 0, k], x0 + (z - a * x0) / 5.0, rtol=1e-13)
        assert np.isclose(s[0, 0, k], 0.3 / 5.0)
