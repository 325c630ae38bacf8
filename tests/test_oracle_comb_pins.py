"""Pins of the oracle's comb-pilot estimators (3W / 12W LMMSE, interpolated LS; Sec. II, IV-B).

Against the group maps the paper prints (Tables I and II), the weight matrices it writes
out (Eq. W1-W3, P), the full LMMSE it reduces to when one window spans every tone, the
LMMSE error closed form under matched statistics, and exactness of the interpolation on
channels it must reproduce.
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


def _span(txt):
    a, st, b = (int(v) for v in txt.split(":"))
    return np.arange(a, b + 1, st)


def _table_i():
    rows = []
    with open(os.path.join(GOLDEN, "eq_w_3w_subscripts.txt")) as f:
        for line in f:
            if line.startswith("group"):
                parts = line.split()
                kv = dict(p.split("=") for p in parts[2:])
                rows.append((int(parts[1]), [int(v) for v in kv["out"].split(",")],
                             int(kv["W"][1:]), [int(v) for v in kv["ls"].split(",")]))
    return rows


def _table_ii():
    rows = []
    with open(os.path.join(GOLDEN, "comb_table_II_12w_groups.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                idx, out, w, ls = line.split()
                rows.append((int(idx), _span(out), int(w), _span(ls)))
    return rows


# ------------------------------------------------------------- group maps (P7)
def test_3w_groups_match_table_i():
    groups = O.comb_groups(O.COMB_3W, 0, 12, 1200)
    tones = O.comb_tones(0, 12, 1200)
    assert len(groups) == 100
    for idx, out, w, ls in _table_i():
        o, i0, widx = groups[idx - 1]
        np.testing.assert_array_equal(o + 1, out)
        np.testing.assert_array_equal(tones[i0:i0 + 3] + 1, ls)
        assert widx + 1 == w


def test_12w_groups_match_table_ii():
    groups = O.comb_groups(O.COMB_SW, 0, 12, 1200)
    tones = O.comb_tones(0, 12, 1200)
    assert len(groups) == 100
    for idx, out, w, ls in _table_ii():
        o, i0, widx = groups[idx - 1]
        np.testing.assert_array_equal(o + 1, out)
        np.testing.assert_array_equal(tones[i0:i0 + 12] + 1, ls)
        assert widx + 1 == w
    # the groups tile every subcarrier once
    allo = np.concatenate([g[0] for g in groups])
    np.testing.assert_array_equal(np.sort(allo), np.arange(1200))


# ----------------------------------------------------------- weights (P6)
def _mats():
    mats, cur = {}, None
    with open(os.path.join(GOLDEN, "eq_w_3w_subscripts.txt")) as f:
        for line in f:
            line = line.strip()
            if line.startswith("matrix"):
                cur = line.split()[1]
                mats[cur] = []
            elif cur and line and not line.startswith(("#", "group")):
                mats[cur].append([int(v) for v in line.split()])
    return {k: np.array(v) for k, v in mats.items()}


@pytest.mark.parametrize("pdp", ["exp", "uniform_L"])
def test_3w_weights_equal_eq_w1_w3_times_inverse_p(pdp):
    """W^(i) = [r at the printed subscripts] (P)^-1 with P = [r_(printed)] + sigma2 I
    (Eq. W1-W3, P; P is inverted as Eq. 17 requires), for groups 1, 2..99 and 100."""
    S, N, s2 = 12, 1200, 0.05
    r = O.make_r("exp", n_taps=8, tau_rms=3.0, n_fft=2048) if pdp == "exp" else \
        O.make_r("uniform_L", L=8.0, n=2048)
    mats = _mats()
    Pm = r(mats["P"].astype(float)) + s2 * np.eye(3)
    tones = O.comb_tones(0, S, N)
    for j, name in ((0, "W1"), (1, "W2"), (50, "W2"), (98, "W2"), (99, "W3")):
        o, i0, _ = O.comb_groups(O.COMB_3W, 0, S, N)[j]
        got = O.comb_weight(o, tones[i0:i0 + 3], r, s2)
        want = r(mats[name].astype(float)) @ np.linalg.inv(Pm)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)


def test_weight_sharing_claims_of_sec_iv_b():
    """3W: three weight matrices shared by every user; 12W: twelve per user, differing
    between users, interior groups sharing one."""
    S, N, s2 = 12, 1200, 0.1
    r = O.make_r("exp", n_taps=6, tau_rms=4.0, n_fft=2048)

    def weights(method, k):
        tones = O.comb_tones(k, S, N)
        Q = 3 if method == O.COMB_3W else S
        out = {}
        for o, i0, widx in O.comb_groups(method, k, S, N):
            out.setdefault(widx, []).append(O.comb_weight(o, tones[i0:i0 + Q], r, s2))
        return out

    w3 = [weights(O.COMB_3W, k) for k in (0, 5, 11)]
    assert sorted(w3[0]) == [0, 1, 2]
    for widx, ws in w3[0].items():
        for W in ws[1:]:
            np.testing.assert_allclose(W, ws[0], rtol=1e-12, atol=1e-14)
        for other in w3[1:]:
            np.testing.assert_allclose(other[widx][0], ws[0], rtol=1e-12, atol=1e-14)
    w12 = [weights(O.COMB_SW, k) for k in (0, 3)]
    assert sorted(w12[0]) == list(range(12))
    assert len(w12[0][5]) == 89                       # groups 6..94 share W^(6)
    for W in w12[0][5][1:]:
        np.testing.assert_allclose(W, w12[0][5][0], rtol=1e-12, atol=1e-14)
    assert np.abs(w12[0][5][0] - w12[1][5][0]).max() > 1e-3


# -------------------------------------------------- special case: full LMMSE
@pytest.mark.parametrize("method", [O.COMB_SW, O.COMB_3W])
def test_window_spanning_all_tones_is_the_full_lmmse(method):
    """With P = Q tones per user every group's window holds all of them, so each estimate
    is the full LMMSE of Eq. 13 from the user's tones (solved here by an explicit inverse)."""
    S = 6
    Q = 3 if method == O.COMB_3W else S
    N = S * Q
    sh = _shape(M=3, K=4, n_sc=N, n_fft=64, n_taps=4, tau_rms=2.0, snr_db=12.0)
    sf = synth.make_comb_subframe(sh, seed=11, S=S)
    r = O.make_r("exp", n_taps=sh.n_taps, tau_rms=sh.tau_rms, n_fft=sh.n_fft)
    h_ls = O.comb_ls(sf["y_pilot"], sf["pilots"], sh.K, S)
    got = O.comb_lmmse(h_ls, method, S, N, r, sh.sigma2)
    for k in range(sh.K):
        tones = O.comb_tones(k, S, N)
        A = r(tones[:, None] - tones[None, :].astype(float)) + sh.sigma2 * np.eye(len(tones))
        if method == O.COMB_SW:
            pos = np.arange(N)
        else:
            pos = (k + np.arange(Q)[:, None] * S + np.arange(3)[None, :] * (S // 3)).ravel()
        R = r(pos[:, None].astype(float) - tones[None, :])
        est = h_ls[:, k] @ (R @ np.linalg.inv(A)).T
        if method == O.COMB_SW:
            np.testing.assert_allclose(got[:, k], est, rtol=1e-11, atol=1e-12)
        else:
            for n in range(N):
                i = max(0, int(np.searchsorted(pos, n, side="right")) - 1)
                np.testing.assert_allclose(got[:, k, :, n], est[..., i], rtol=1e-11, atol=1e-12)


# -------------------------------------------------------------- LS, hold, interp
def test_comb_ls_noiseless_is_the_channel_on_each_users_tones():
    sh = _shape(M=4, K=3, n_sc=48, n_fft=64)
    sf = synth.make_comb_subframe(sh, seed=2, S=4, noiseless=True)
    h_ls = O.comb_ls(sf["y_pilot"], sf["pilots"], sh.K, 4)
    for k in range(sh.K):
        tn = O.comb_tones(k, 4, sh.n_sc)
        np.testing.assert_allclose(h_ls[:, k], np.broadcast_to(sf["H"][:, k, tn], h_ls[:, k].shape),
                                   rtol=1e-13, atol=1e-14)


def test_interp3_reproduces_a_linear_channel_and_holds():
    S, N, P = 12, 96, 8
    n = np.arange(N)
    K = 2
    H = np.stack([(0.3 - 0.2j) + (0.01 + 0.02j) * n, (1.1 + 0.4j) - 0.015j * n])      # [K][N]
    h_ls = np.stack([H[k, O.comb_tones(k, S, N)] for k in range(K)])[None, :, None, :]
    got = O.comb_interp3_ls(h_ls, S, N)[0, :, 0]
    for k in range(K):
        for v in range(3 * (P - 1)):                  # grid points between the first and last tone
            q = k + v * (S // 3)
            np.testing.assert_allclose(got[k, q], H[k, q], rtol=1e-13, atol=1e-13)
            np.testing.assert_allclose(got[k, q:q + S // 3], got[k, q], rtol=0, atol=0)
        np.testing.assert_allclose(got[k, :k + 1], H[k, k], rtol=1e-13)
        np.testing.assert_allclose(got[k, k + (P - 1) * S:], H[k, k + (P - 1) * S], rtol=1e-13)


# ------------------------------------------------- matched statistics (MC)
def test_12w_error_matches_lmmse_theory_monte_carlo():
    """Matched model: E|h^ - h|^2 at output u of a group = [R_oo - W R_{H Hls}^H]_uu."""
    S, N = 6, 72
    sh = _shape(M=24, K=3, n_sc=N, n_fft=128, n_taps=5, tau_rms=3.0, snr_db=8.0)
    r = O.make_r("exp", n_taps=sh.n_taps, tau_rms=sh.tau_rms, n_fft=sh.n_fft)
    errs = []
    for seed in range(5):
        sf = synth.make_comb_subframe(sh, seed=40 + seed, S=S)
        h_ls = O.comb_ls(sf["y_pilot"], sf["pilots"], sh.K, S)
        h = O.comb_lmmse(h_ls, O.COMB_SW, S, N, r, sh.sigma2)
        errs.append(np.abs(h - np.transpose(sf["H"], (1, 0, 2))[None]) ** 2)
    e = np.concatenate(errs, axis=0)                  # [runs*T][K][M][N]
    theory = np.empty((sh.K, N))
    for k in range(sh.K):
        tones = O.comb_tones(k, S, N)
        for o, i0, _ in O.comb_groups(O.COMB_SW, k, S, N):
            t = tones[i0:i0 + S]
            W = O.comb_weight(o, t, r, sh.sigma2)
            Rot = O.corr_matrix(o, t, r)
            theory[k, o] = np.real(1.0 - np.einsum("ui,ui->u", W, Rot.conj()))
    got = e.mean(axis=(0, 2))
    se = e.std(axis=(0, 2)) / np.sqrt(e.shape[0] * e.shape[2])
    # per user: the subcarrier-averaged error against theory, within 4 standard errors
    # (the per-subcarrier errors of one run are correlated, so the bound uses their spread)
    for k in range(sh.K):
        assert abs(got[k].mean() - theory[k].mean()) < 4 * se[k].mean(), (k, got[k].mean(), theory[k].mean())
    assert np.all(np.abs(got - theory) < 5 * se)


def test_comb_estimator_gaps_of_fig_7a():
    """Sec. V on Fig. 7(a) (Table III: 16 antennas, 4 users on a comb of 12, 1200 of 2048
    subcarriers, taps at delays 0..5 with powers -2, -8, -10, -12, -15, -18 dB; weights for
    L = 8 and SNR_fixed = 40 dB): 12W gains about 7 dB over LS and stays about 3 dB from
    the full LMMSE; 3W gains about 3.8 dB over LS and 2 dB over three-fold interpolated LS.
    LS is scored on the pilot tones it estimates; the rest on every subcarrier."""
    S, N = 12, 1200
    sh = _shape(M=16, K=4, n_sc=N, n_fft=2048, snr_db=20.0, qam_bits=6)
    tap_db = np.array([-2.0, -8.0, -10.0, -12.0, -15.0, -18.0])
    r = O.make_r("uniform_L", L=8.0, n=2048)
    s2_fixed = 10 ** (-40 / 10)
    sf = synth.make_comb_subframe(sh, seed=7, S=S, tap_powers=10 ** (tap_db / 10))
    H = np.transpose(sf["H"], (1, 0, 2))[None]
    h_ls = O.comb_ls(sf["y_pilot"], sf["pilots"], sh.K, S)
    db = lambda e: 10 * np.log10(np.mean(np.abs(e) ** 2))
    ls = db(np.stack([h_ls[:, k] - H[:, k][..., O.comb_tones(k, S, N)] for k in range(sh.K)], axis=1))
    w12 = db(O.comb_lmmse(h_ls, O.COMB_SW, S, N, r, s2_fixed) - H)
    w3 = db(O.comb_lmmse(h_ls, O.COMB_3W, S, N, r, s2_fixed) - H)
    interp = db(O.comb_interp3_ls(h_ls, S, N) - H)
    full = db(np.stack([h_ls[:, k] @ O.comb_weight(np.arange(N), O.comb_tones(k, S, N), r, s2_fixed).T
                        - H[:, k] for k in range(sh.K)], axis=1))
    gaps = dict(w12_vs_ls=ls - w12, full_vs_w12=w12 - full, w3_vs_ls=ls - w3, w3_vs_interp=interp - w3)
    want = dict(w12_vs_ls=7.0, full_vs_w12=3.0, w3_vs_ls=3.8, w3_vs_interp=2.0)
    for k, v in want.items():
        assert abs(gaps[k] - v) < 0.75, gaps
