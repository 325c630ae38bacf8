"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a value the paper
prints, a closed form computed by a different route (eigendecomposition, SVD least
squares, the M x M push-through form), a brute-force search, or a Monte-Carlo
statistic of the generator's channel law.
"""
import os

import numpy as np
import pytest

from oracle import rapro_oracle as O
from paper_1802_05427_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _shape(**kw):
    base = dict(M=8, K=2, n_sc=72, n_fft=128, n_taps=6, tau_rms=4.0, snr_db=10.0, qam_bits=2)
    base.update(kw)
    return synth.SubframeShape(**base)


# ------------------------------------------------------------------ P1: LS
def test_ls_noiseless_equals_true_channel():
    """Eq. 9: without noise, Y/X returns H exactly, for unit and non-unit pilots."""
    sh = _shape(M=4, K=3, n_sc=40)
    rng = np.random.default_rng(3)
    mod = rng.uniform(0.5, 2.0, size=(sh.n_slots, sh.K, sh.n_sc))
    for pm in (None, mod):
        sf = synth.make_subframe(sh, seed=11, noiseless=True, pilot_modulus=pm)
        h_ls = O.ls_estimate(sf["y_pilot"], sf["pilots"])
        truth = np.transpose(sf["H"], (1, 0, 2))[None]            # [1][K][M][N]
        np.testing.assert_allclose(h_ls, np.broadcast_to(truth, h_ls.shape), rtol=0, atol=1e-14)


# ------------------------------------------------------ correlation models
def test_uniform_L_correlation_properties():
    """Eq. 16: r(0)=1, Hermitian symmetry, |r|<=1, zeros where L d / N is a nonzero integer,
    and equality with the average of exp(-j 2 pi tau d / N) over tau in [0, L]."""
    L, N = 8.0, 2048.0
    d = np.arange(-300, 301)
    r = O.corr_uniform_L(d, L, N)
    assert r[300] == 1.0
    np.testing.assert_allclose(r[::-1], np.conj(r), atol=1e-15)
    assert np.all(np.abs(r) <= 1 + 1e-15)
    for z in (256, -256, 512):
        assert abs(O.corr_uniform_L(np.array([z]), L, N)[0]) < 1e-14
    # midpoint rule over the uniform delay law (an independent route to Eq. 16)
    tau = (np.arange(200000) + 0.5) / 200000 * L
    for dd in (1, 7, 33, -120):
        avg = np.mean(np.exp(-2j * np.pi * tau * dd / N))
        assert abs(avg - O.corr_uniform_L(np.array([dd]), L, N)[0]) < 1e-9


def test_exponential_correlation_matches_generator_channel():
    """r(d) = E{H(k+d) H(k)^*} for the generator's channel law, by Monte Carlo.

    Pins the sign of the phase (a conjugated r would fail) and the normalisation."""
    sh = _shape(M=64, K=8, n_sc=64, n_taps=6, tau_rms=2.0)
    acc = {d: 0.0 for d in (0, 1, 3, 9, -5)}
    n = 0
    for seed in range(4):
        H = synth.make_subframe(sh, seed=100 + seed, noiseless=True)["H"]  # [M][K][N]
        for d in acc:
            if d >= 0:
                prod = H[:, :, d:] * np.conj(H[:, :, :sh.n_sc - d])
            else:
                prod = H[:, :, :sh.n_sc + d] * np.conj(H[:, :, -d:])
            acc[d] += prod.mean() * 1.0
        n += 1
    for d, v in acc.items():
        r = O.corr_exponential(np.array([d]), sh.n_taps, sh.tau_rms, sh.n_fft)[0]
        assert abs(v / n - r) < 0.03, (d, v / n, r)
    assert abs(O.corr_exponential(np.array([0]), 24, 8.0, 2048)[0] - 1.0) < 1e-14
    one_tap = O.corr_exponential(np.arange(-50, 50), 1, 3.0, 2048)
    np.testing.assert_allclose(one_tap, 1.0, atol=1e-15)


def _read_golden():
    groups, mats, cur = [], {}, None
    with open(os.path.join(GOLDEN, "eq_w_3w_subscripts.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("group"):
                parts = dict(p.split("=") for p in line.split()[2:])
                groups.append(([int(v) for v in parts["out"].split(",")],
                               [int(v) for v in parts["ls"].split(",")], parts["W"]))
            elif line.startswith("matrix"):
                cur = line.split()[1]
                mats[cur] = []
            else:
                mats[cur].append([int(v) for v in line.split()])
    return groups, {k: np.array(v) for k, v in mats.items()}


def test_corr_matrix_index_convention_worked_3w_example():
    """Eq. W1-W3 and P with the Table I groups: entry (a, b) is r at k_out[a] - k_ls[b]."""
    groups, mats = _read_golden()
    ident = lambda d: d                            # r_d -> d shows which subscript is used
    for out, ls, wname in groups:
        got = O.corr_matrix(out, ls, ident).astype(int)
        np.testing.assert_array_equal(got, mats[wname])
        got_p = O.corr_matrix(ls, ls, ident).astype(int)
        np.testing.assert_array_equal(got_p, mats["P"])


# ------------------------------------------------------------- P2: weights
@pytest.mark.parametrize("B", [1, 5, 12, 48])
@pytest.mark.parametrize("sigma2", [1.0, 0.1, 0.01])
def test_lmmse_weight_closed_forms(B, sigma2):
    """W = R (R + s I)^-1 is Hermitian with eigenvalues l/(l+s), and W = I - s (R + s I)^-1."""
    r = O.make_r("exp", n_taps=24, tau_rms=8.0, n_fft=2048)
    idx = np.arange(B)
    R = O.corr_matrix(idx, idx, r)
    W = O.lmmse_weight(R, R, sigma2)
    lam, V = np.linalg.eigh(R)
    W_eig = (V * (lam / (lam + sigma2))) @ V.conj().T
    np.testing.assert_allclose(W, W.conj().T, atol=1e-12)
    np.testing.assert_allclose(W, W_eig, atol=1e-11)
    np.testing.assert_allclose(W, np.eye(B) - (V * (sigma2 / (lam + sigma2))) @ V.conj().T, atol=1e-11)
    if B == 1:
        assert abs(W[0, 0] - 1.0 / (1.0 + sigma2)) < 1e-15


def test_uniform_L_weights_scalar_block():
    """B = 1 under the paper's Eq. 16 model: r(0) = 1 so w = 1 / (1 + sigma2)."""
    r = O.make_r("uniform_L", L=8.0, n=2048.0)
    W = O.subblock_weights(5, 1, r, 0.25)
    for _, w in W:
        assert abs(w[0, 0] - 0.8) < 1e-15


# ---------------------------------------------------- P3: full vs sub-block
def test_subblock_with_block_spanning_all_subcarriers_equals_full_lmmse():
    """B = N_sc is the full LMMSE of Eq. 13; computed here independently by eigh."""
    sh = _shape(M=4, K=2, n_sc=96, n_fft=256, n_taps=8, tau_rms=3.0, snr_db=5.0)
    sf = synth.make_subframe(sh, seed=5)
    h_ls = O.ls_estimate(sf["y_pilot"], sf["pilots"])
    r = O.make_r("exp", n_taps=sh.n_taps, tau_rms=sh.tau_rms, n_fft=sh.n_fft)
    got = O.subblock_lmmse(h_ls, sh.n_sc, r, sh.sigma2)
    idx = np.arange(sh.n_sc)
    lam, V = np.linalg.eigh(O.corr_matrix(idx, idx, r))
    W = (V * (lam / (lam + sh.sigma2))) @ V.conj().T
    np.testing.assert_allclose(got, h_ls @ W.T, rtol=0, atol=1e-10)


def test_subblocks_are_independent_and_tail_has_own_weight():
    """Non-overlapping blocks (Eq. 12 per block): a change inside one block stays there;
    the last block of N_sc mod B subcarriers is filtered by its own smaller W."""
    r = O.make_r("exp", n_taps=6, tau_rms=4.0, n_fft=128)
    rng = np.random.default_rng(0)
    h = rng.standard_normal((1, 1, 2, 30)) + 1j * rng.standard_normal((1, 1, 2, 30))
    base = O.subblock_lmmse(h, 12, r, 0.1)
    h2 = h.copy()
    h2[..., 13] += 1.0
    pert = O.subblock_lmmse(h2, 12, r, 0.1)
    changed = np.any(np.abs(pert - base) > 0, axis=(0, 1, 2))
    assert changed[12:24].all() and not changed[:12].any() and not changed[24:].any()
    idx = np.arange(6)
    lam, V = np.linalg.eigh(O.corr_matrix(idx, idx, r))
    Wt = (V * (lam / (lam + 0.1))) @ V.conj().T
    np.testing.assert_allclose(base[..., 24:], h[..., 24:] @ Wt.T, atol=1e-12)


# ------------------------------------------------ P4: noiseless projection
def test_lmmse_preserves_noiseless_channel_in_model_range():
    """With matched statistics the channel lies in range(R_b) (a sum of n_taps steering
    vectors), so W_b -> projection as sigma2 -> 0 and W_b H = H."""
    sh = _shape(M=4, K=2, n_sc=96, n_fft=128, n_taps=6, tau_rms=4.0)
    H = np.transpose(synth.make_subframe(sh, seed=9, noiseless=True)["H"], (1, 0, 2))[None]
    r = O.make_r("exp", n_taps=sh.n_taps, tau_rms=sh.tau_rms, n_fft=sh.n_fft)
    for B in (12, 48, 96):
        got = O.subblock_lmmse(H, B, r, 1e-12)
        err = np.linalg.norm(got - H) / np.linalg.norm(H)
        assert err < 1e-4, (B, err)


# ----------------------------------------------- P5: MSE of matched LMMSE
def test_lmmse_mse_matches_theory_monte_carlo():
    """Matched statistics: E|H^ - H|^2 per subcarrier = sigma2 tr(W_b) / B_b; LS gives sigma2."""
    sh = _shape(M=32, K=4, n_sc=48, n_fft=128, n_taps=6, tau_rms=4.0, snr_db=3.0)
    r = O.make_r("exp", n_taps=sh.n_taps, tau_rms=sh.tau_rms, n_fft=sh.n_fft)
    B = 12
    errs, errs_ls = [], []
    for seed in range(6):
        sf = synth.make_subframe(sh, seed=300 + seed)
        H = np.transpose(sf["H"], (1, 0, 2))[None]
        h_ls = O.ls_estimate(sf["y_pilot"], sf["pilots"])
        h = O.subblock_lmmse(h_ls, B, r, sh.sigma2)
        errs.append((np.abs(h - H) ** 2).ravel())
        errs_ls.append((np.abs(h_ls - H) ** 2).ravel())
    e, e_ls = np.concatenate(errs), np.concatenate(errs_ls)
    W = O.subblock_weights(B, B, r, sh.sigma2)[0][1]
    theory = sh.sigma2 * np.real(np.trace(W)) / B
    se = e.std() / np.sqrt(e.size) * 4          # generous: samples are correlated within blocks
    assert abs(e.mean() - theory) < 4 * se, (e.mean(), theory, se)
    assert abs(e_ls.mean() - sh.sigma2) < 4 * e_ls.std() / np.sqrt(e_ls.size) * 2
    assert e.mean() < 0.5 * e_ls.mean()


# ------------------------------------------------------- P8 / P12: detection
def _detect_inputs(M, K, N, D, seed, snr_db=20.0, q=2):
    sh = _shape(M=M, K=K, n_sc=N, n_data_per_slot=D, snr_db=snr_db, qam_bits=q)
    sf = synth.make_subframe(sh, seed=seed)
    h = np.broadcast_to(np.transpose(sf["H"], (1, 0, 2))[None], (sh.n_slots, K, M, N)).copy()
    return sh, sf, h


def test_mmse_tends_to_zero_forcing_and_recovers_noiseless_symbols():
    """Eq. 19 vs Eq. 21: sigma2 -> 0 gives the pseudo-inverse (SVD least squares);
    with the true channel and no noise, x~ = x."""
    M, K, N, D = 6, 3, 10, 6
    sh, sf, h = _detect_inputs(M, K, N, D, seed=21)
    x, _ = O.mmse_detect(h, sf["y_data"], 1e-13, D)
    for n in (0, 7):
        for k in (0, 9):
            Hk = sf["H"][:, :, k]
            ref = np.linalg.lstsq(Hk, sf["y_data"][n, :, k], rcond=None)[0]
            np.testing.assert_allclose(x[n, :, k], ref, atol=1e-9)
    sf0 = synth.make_subframe(sh, seed=21, noiseless=True)
    x0, _ = O.mmse_detect(h, sf0["y_data"], 0.0, D)
    np.testing.assert_allclose(x0, sf0["x"], atol=1e-12)


def test_mmse_push_through_form():
    """x~ = (H^H H + s I)^-1 H^H y equals H^H (H H^H + s I)^-1 y (M x M form)."""
    M, K, N, D = 5, 3, 7, 6
    sh, sf, h = _detect_inputs(M, K, N, D, seed=4, snr_db=3.0)
    s2 = 0.37
    x, s = O.mmse_detect(h, sf["y_data"], s2, D)
    for k in range(N):
        Hk = sf["H"][:, :, k]
        G = Hk.conj().T @ np.linalg.inv(Hk @ Hk.conj().T + s2 * np.eye(M))
        for n in (0, 6, 11):
            np.testing.assert_allclose(x[n, :, k], G @ sf["y_data"][n, :, k], atol=1e-12)
        # mu_k = [A^-1 H^H H]_kk from the eigendecomposition of H^H H
        lam, V = np.linalg.eigh(Hk.conj().T @ Hk)
        mu = np.real(np.diagonal((V * (lam / (lam + s2))) @ V.conj().T))
        np.testing.assert_allclose(1.0 - s[0, :, k], mu, atol=1e-12)


def test_mmse_single_user_scalar_form():
    """K = 1: x~ = h^H y / (|h|^2 + s) and s [A^-1] = s / (|h|^2 + s) (textbook scalar MMSE)."""
    M, N, D = 7, 9, 6
    sh, sf, h = _detect_inputs(M, 1, N, D, seed=8)
    s2 = 0.2
    x, s = O.mmse_detect(h, sf["y_data"], s2, D)
    Hm = sf["H"][:, 0, :]                                      # [M][N]
    g = np.sum(np.abs(Hm) ** 2, axis=0)
    ref = np.einsum("mn,dmn->dn", np.conj(Hm), sf["y_data"]) / (g + s2)
    np.testing.assert_allclose(x[:, 0, :], ref, atol=1e-13)
    np.testing.assert_allclose(s[0, 0], s2 / (g + s2), atol=1e-15)


def test_unbiased_estimate_by_monte_carlo():
    """E{x~_k | x} = mu_k x_k with mu_k = 1 - sigma2 [A^-1]_kk (noise averaged out)."""
    rng = np.random.default_rng(1)
    M, K, s2 = 4, 2, 0.5
    Hk = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) / np.sqrt(2)
    x = np.array([1 + 1j, -1 + 1j]) / np.sqrt(2)
    T = 20000
    noise = np.sqrt(s2 / 2) * (rng.standard_normal((M, T)) + 1j * rng.standard_normal((M, T)))
    y = (Hk @ x)[:, None] + noise                               # [M][T]
    h = np.transpose(Hk, (1, 0))[None, :, :, None].repeat(T, axis=3)  # [1][K][M][T]
    xe, s = O.mmse_detect(h, y[None], s2, 1)
    mu = 1.0 - s[0, :, 0]
    np.testing.assert_allclose(xe[0].mean(axis=1), mu * x, atol=0.02)


def test_unbiased_estimate_and_nu_single_user_closed_form():
    """K = 1: x^ = x~ / mu = h^H y / |h|^2 (unbiased matched filter) and nu = sigma2 / |h|^2."""
    M, N, D = 5, 11, 6
    sh, sf, h = _detect_inputs(M, 1, N, D, seed=13)
    s2 = 0.3
    x, s = O.mmse_detect(h, sf["y_data"], s2, D)
    xhat, nu = O.unbias(x, s, D)
    Hm = sf["H"][:, 0, :]
    g = np.sum(np.abs(Hm) ** 2, axis=0)
    np.testing.assert_allclose(xhat[:, 0, :], np.einsum("mn,dmn->dn", np.conj(Hm), sf["y_data"]) / g,
                               atol=1e-12)
    np.testing.assert_allclose(nu[:, 0, :], np.broadcast_to(s2 / g, (sh.n_data, N)), rtol=1e-12)


def test_nu_is_error_variance_of_unbiased_estimate_monte_carlo():
    """For unit-energy i.i.d. symbols, Var{x^_k - x_k} = nu_k = (1 - mu_k) / mu_k."""
    rng = np.random.default_rng(6)
    M, K, s2, T = 4, 3, 0.4, 40000
    Hk = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) / np.sqrt(2)
    x = O.constellation(2)[rng.integers(0, 4, size=(K, T))]
    noise = np.sqrt(s2 / 2) * (rng.standard_normal((M, T)) + 1j * rng.standard_normal((M, T)))
    y = Hk @ x + noise
    h = np.transpose(Hk, (1, 0))[None, :, :, None].repeat(T, axis=3)
    xe, s = O.mmse_detect(h, y[None], s2, 1)
    xhat, nu = O.unbias(xe, s, 1)
    var = np.mean(np.abs(xhat[0] - x) ** 2, axis=1)
    np.testing.assert_allclose(var, nu[0, :, 0], rtol=0.05)


# ------------------------------------------------------- P9: brute-force ML
@pytest.mark.parametrize("K", [2, 3])
def test_mmse_agrees_with_brute_force_ml_at_high_snr(K):
    """ML over all 4^K QPSK vectors; MMSE hard decisions agree on >= 99.9% of REs at 30 dB,
    and at 5 dB MMSE makes at least as many symbol errors as ML."""
    M, N, D = 4, 200, 6
    pts = O.constellation(2)
    cands = np.array(np.meshgrid(*([np.arange(4)] * K), indexing="ij")).reshape(K, -1).T
    for snr, check in ((30.0, "agree"), (5.0, "ml_better")):
        sh, sf, h = _detect_inputs(M, K, N, D, seed=40 + K, snr_db=snr)
        x, s = O.mmse_detect(h, sf["y_data"], sh.sigma2, D)
        xhat, _ = O.unbias(x, s, D)
        lab = O.hard_decision(xhat, 2)
        ml = np.empty_like(lab)
        for k in range(N):
            Hk = sf["H"][:, :, k]
            X = pts[cands].T                                   # [K][C]
            d = np.abs(sf["y_data"][:, :, k][:, :, None] - (Hk @ X)[None]) ** 2
            ml[:, :, k] = cands[np.argmin(d.sum(axis=1), axis=1)]
        if check == "agree":
            assert np.mean(np.all(lab == ml, axis=1)) >= 0.999
        else:
            assert np.sum(lab != sf["labels"]) >= np.sum(ml != sf["labels"])


# ------------------------------------------------------------ P11: demapper
@pytest.mark.parametrize("q", [2, 4, 6])
def test_constellation_gray_unit_energy_and_roundtrip(q):
    pts = O.constellation(q)
    assert abs(np.mean(np.abs(pts) ** 2) - 1.0) < 1e-14
    labels = np.arange(1 << q)
    np.testing.assert_allclose(synth.gray_qam_map(labels, q), pts, atol=1e-15)
    np.testing.assert_array_equal(O.hard_decision(pts, q), labels)
    dmin = np.min(np.abs(pts[:, None] - pts[None, :]) + 10 * np.eye(1 << q))
    for a in range(1 << q):
        for b in range(1 << q):
            if abs(abs(pts[a] - pts[b]) - dmin) < 1e-12:
                assert bin(a ^ b).count("1") == 1      # Gray: nearest neighbours differ in one bit
    # the leading I bit (b0) and leading Q bit (b1) select the positive half at value 0
    assert np.all((np.real(pts) > 0) == (((labels >> (q - 1)) & 1) == 0))
    assert np.all((np.imag(pts) > 0) == (((labels >> (q - 2)) & 1) == 0))


def test_llr_closed_forms_and_signs():
    rng = np.random.default_rng(2)
    xhat = rng.standard_normal(500) + 1j * rng.standard_normal(500)
    nu = rng.uniform(0.05, 1.0, 500)
    # QPSK: levels +-1/sqrt2 per dimension -> LLR = 2 sqrt(2) x / nu
    llr = O.maxlog_llr(xhat, nu, 2)
    np.testing.assert_allclose(llr[:, 0], 2 * np.sqrt(2) * np.real(xhat) / nu, rtol=1e-12)
    np.testing.assert_allclose(llr[:, 1], 2 * np.sqrt(2) * np.imag(xhat) / nu, rtol=1e-12)
    # 16-QAM leading bit on [0, 2/sqrt10]: nearest 0-point 1/sqrt10, nearest 1-point -1/sqrt10
    xs = np.linspace(0.0, 2.0 / np.sqrt(10), 7) + 0.1j
    l16 = O.maxlog_llr(xs, np.ones(7), 4)
    np.testing.assert_allclose(l16[:, 0], 4 * np.real(xs) / np.sqrt(10), atol=1e-12)
    for q in (2, 4, 6):
        lab = O.hard_decision(xhat * 0.7, q)
        ll = O.maxlog_llr(xhat * 0.7, nu, q)
        for i in range(q):
            bit = (lab >> (q - 1 - i)) & 1
            nz = np.abs(ll[:, i]) > 1e-9
            assert np.all((ll[nz, i] > 0) == (bit[nz] == 0))


def _pam_maxlog_closed_form(y, s0):
    """Max-log LLR of one Gray PAM bit on the integer grid (levels odd integers), written as
    the exact piecewise-linear forms of the Gray 4- and 8-PAM demappers; s0 = the levels
    where the bit is 0.  Returns None for a level set that is not one of those forms."""
    a = np.abs(y)
    sg = np.sign(y)
    s0 = frozenset(s0)
    forms = {
        # 4-PAM (16-QAM per dimension)
        frozenset({1, 3}): np.where(a <= 2, 4 * y, 8 * (y - sg)),
        frozenset({-1, 1}): 4 * (2 - a),
        # 8-PAM (64-QAM per dimension)
        frozenset({1, 3, 5, 7}): np.select([a <= 2, a <= 4, a <= 6],
                                           [4 * y, 8 * (y - sg), 12 * (y - 2 * sg)], 16 * (y - 3 * sg)),
        frozenset({-3, -1, 1, 3}): np.select([a <= 2, a <= 6], [8 * (3 - a), 4 * (4 - a)], 8 * (5 - a)),
        frozenset({-7, -1, 1, 7}): 4 * (np.abs(a - 4) - 2),
    }
    if s0 in forms:
        return forms[s0]
    levels = frozenset(range(-7, 8, 2)) if max(s0) > 3 or min(s0) < -3 else frozenset({-3, -1, 1, 3})
    comp = levels - s0
    if comp in forms:
        return -forms[comp]
    return None


@pytest.mark.parametrize("q", [4, 6])
def test_llr_matches_gray_pam_piecewise_linear_forms(q):
    """Every bit of the 16- and 64-QAM max-log LLR against the exact per-dimension piecewise
    linear forms of Gray PAM (Eq. 22 read as max-log over the product constellation)."""
    m = q // 2
    scale = np.sqrt(2.0 * (4 ** m - 1) / 3.0)          # unit mean energy: levels / scale
    rng = np.random.default_rng(11 + q)
    y = rng.uniform(-(1 << m) - 2, (1 << m) + 2, (2, 3000))
    xhat = (y[0] + 1j * y[1]) / scale
    nu = rng.uniform(0.05, 2.0, 3000)
    llr = O.maxlog_llr(xhat, nu, q)
    pts = O.constellation(q)
    labels = np.arange(1 << q)
    for i in range(q):
        bit = (labels >> (q - 1 - i)) & 1
        for dim, part in enumerate((np.real, np.imag)):
            lv = np.rint(part(pts) * scale).astype(int)
            if all(len(set(bit[lv == v])) == 1 for v in set(lv)):   # this bit lives on `dim`
                s0 = {int(v) for v in set(lv[bit == 0])}
                f = _pam_maxlog_closed_form(y[dim], s0)
                assert f is not None, (q, i, s0)
                np.testing.assert_allclose(llr[:, i], f / (scale ** 2 * nu), rtol=1e-11, atol=1e-11)
                break
        else:
            raise AssertionError(f"bit {i} of {q}-bit labels depends on both dimensions")


def test_boundary_margin_units():
    for q in (2, 4, 6):
        pts = O.constellation(q)
        np.testing.assert_allclose(O.boundary_margin(pts, q), 1.0, atol=1e-12)
    assert O.boundary_margin(np.array([0.0 + 0.5j]), 2)[0] == 0.0


# Off-lattice points in lattice units (levels on the odd integers, d_min / 2 = 1), with the
# distance to the nearest decision boundary worked out by hand.  Boundaries per dimension:
# QPSK {0}; 16-QAM {-2, 0, 2}; 64-QAM {-6, -4, -2, 0, 2, 4, 6}.  Each row: (I, Q, margin).
_MARGIN_CASES = {
    2: [(0.3, -0.8, 0.3), (-2.0, 1.5, 1.5), (0.9, 0.05, 0.05)],
    4: [(0.3, 2.9, 0.3),          # I 0.3 from 0; Q 0.9 from 2
        (-1.6, 0.55, 0.4),        # I 0.4 from -2; Q 0.55 from 0
        (3.8, -3.5, 1.5),         # outer cell: I 1.8 from 2, Q 1.5 from -2
        (0.05, -1.0, 0.05),       # the interior boundary at 0 decides it (else 1.0)
        (2.25, 1.1, 0.25),        # I 0.25 from 2; Q 0.9 from 2
        (-1.0, -0.2, 0.2)],       # Q 0.2 from 0 (else 1.0, from I)
    6: [(0.1, 6.9, 0.1),          # I 0.1 from 0; Q 0.9 from 6
        (-4.7, 3.2, 0.7),         # I 0.7 from -4; Q 0.8 from 4
        (5.35, -2.6, 0.6),        # I 0.65 from 6; Q 0.6 from -2
        (-9.0, -0.45, 0.45),      # I 3 from -6; Q 0.45 from 0
        (3.05, 1.02, 0.95),       # I 0.95 from 4; Q 0.98 from 2
        (-0.3, 5.0, 0.3)],        # I 0.3 from 0 (else 1.0, from Q's 4 and 6)
}


def _margin_cases(q):
    scale = np.sqrt(2.0 * (4 ** (q // 2) - 1) / 3.0)
    c = np.array(_MARGIN_CASES[q])
    return (c[:, 0] + 1j * c[:, 1]) / scale, c[:, 2]


@pytest.mark.parametrize("q", [2, 4, 6])
def test_boundary_margin_off_lattice_by_hand(q):
    x, want = _margin_cases(q)
    np.testing.assert_allclose(O.boundary_margin(x, q), want, atol=1e-12)


def test_boundary_margin_pin_rejects_a_dropped_interior_boundary():
    """The hand-worked table fails a margin whose boundary set misses the one at 0."""
    def margin_without_zero(xhat, q):
        m = q // 2
        scale = np.sqrt(2.0 * (4 ** m - 1) / 3.0)
        bounds = np.array([b for b in range(-(1 << m) + 2, (1 << m) - 1, 2) if b != 0], dtype=float)
        if bounds.size == 0:
            return np.full(xhat.shape, np.inf)
        d = [np.min(np.abs(c[..., None] * scale - bounds), axis=-1) for c in (np.real(xhat), np.imag(xhat))]
        return np.minimum(d[0], d[1])
    for q in (4, 6):
        x, want = _margin_cases(q)
        assert not np.allclose(margin_without_zero(x, q), want, atol=1e-12)


# ------------------------------------------------------ end-to-end sanity
def test_receive_chain_high_snr_is_error_free_and_lmmse_beats_ls():
    sh = _shape(M=16, K=4, n_sc=96, n_fft=256, n_taps=6, tau_rms=4.0, snr_db=25.0, qam_bits=4)
    sf = synth.make_subframe(sh, seed=77)
    r = O.make_r("exp", n_taps=sh.n_taps, tau_rms=sh.tau_rms, n_fft=sh.n_fft)
    out = O.receive_subframe(sf["y_pilot"], sf["pilots"], sf["y_data"], B=12, sigma2=sh.sigma2,
                             r=r, n_data_per_slot=sh.n_data_per_slot, q=sh.qam_bits)
    np.testing.assert_array_equal(out["labels"], sf["labels"])
    H = np.transpose(sf["H"], (1, 0, 2))[None]
    nmse = lambda a: np.sum(np.abs(a - H) ** 2) / np.sum(np.abs(np.broadcast_to(H, a.shape)) ** 2)
    assert nmse(out["h"]) < 0.5 * nmse(out["h_ls"])
