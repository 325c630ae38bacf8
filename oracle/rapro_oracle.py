"""Plain FP64 CPU oracle of the uplink receive path: LS -> sub-block LMMSE -> MMSE detection.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  It shares no code with the CUDA library
(no kernels, headers, tables or helpers); both read the same seeded inputs.

Every function follows the paper's definition directly, in complex128 / float64,
with numpy matmul and LAPACK LU (``numpy.linalg.solve``/``inv``) as the only library
steps.  No blocking, fusion or reordering beyond what each equation states.

Notation (the paper's letters in brackets): M antennas [R], K users [S], N_sc used
subcarriers [N], n_fft FFT size [N_FFT], n_taps channel taps [M], B sub-block size.

Array layouts (the C-ABI layouts, subcarrier index fastest):
  y_pilot, h_ls, h   [T][K][M][N_sc]   T = pilot symbols = slots
  pilots             [T][K][N_sc]
  y_data             [T*D][M][N_sc]    D data symbols per slot, slot of data symbol n = n // D
  x_eq               [T*D][K][N_sc]
  labels (hard)      [T*D][K][N_sc]    Gray label, b0 = most significant of the q bits
  llr                [T*D][K][N_sc][q]

Readings of points the paper leaves open (each also listed in the design notes):
  * pilots are per-user orthogonal observations (one per user and slot), so LS gives
    an estimate on every subcarrier and R_{H Hls} = R_{HH} (Eq. 14/15 with white noise);
  * the frequency correlation uses the FFT size as the denominator of Eq. 16 (the
    phase of a delay tau on bin k is exp(-j 2 pi tau k / n_fft));
  * the exponential PDP model (Sec. III-A text under Eq. 16) with integer taps gives
    r(d) = sum_l p_l exp(-j 2 pi l d / n_fft), p_l ~ exp(-l / tau_rms), sum p_l = 1;
  * sub-blocks are contiguous and non-overlapping from subcarrier 0; the last one has
    N_sc mod B subcarriers and its own W;
  * comb pilots (3W / 12W, Sec. IV-B): user k on tones k + iS; groups and windows as in
    Tables I and II (the last 12W group is subcarriers 1189..1200 in the paper's 1-based
    numbering: the printed 1190:1:1200 has 11 entries); 3W estimates and the three-fold
    interpolated LS are zero-order held to every subcarrier (Sec. IV-C); past the last
    tone the interpolated LS holds that tone's LS;
  * Gray QAM per dimension, unit mean energy; hard decision = nearest point;
    max-log LLR_i = (min_{b_i=1} |x^ - x|^2 - min_{b_i=0} |x^ - x|^2) / nu with the
    unbiased x^ = x~ / mu, mu_k = 1 - sigma2 [A^-1]_kk, nu = (1 - mu) / mu.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------- LS
def ls_estimate(y_pilot: np.ndarray, pilots: np.ndarray) -> np.ndarray:
    """Eq. 8-9: H_LS(k) = Y(k) / X(k) on every pilot tone, per (slot, user, antenna).

    Written as Y conj(X) / |X|^2, which is Y / X exactly in exact arithmetic.
    """
    y = np.asarray(y_pilot, dtype=np.complex128)
    p = np.asarray(pilots, dtype=np.complex128)[:, :, None, :]
    return y * np.conj(p) / (np.abs(p) ** 2)


# ------------------------------------------------------- frequency correlation
def corr_uniform_L(d, L: float, n: float) -> np.ndarray:
    """Eq. 16 / r_d: r(0) = 1, r(d) = (1 - exp(-j 2 pi L d / n)) / (j 2 pi L d / n)."""
    d = np.asarray(d, dtype=np.float64)
    out = np.ones(d.shape, dtype=np.complex128)
    nz = d != 0
    arg = 2j * np.pi * L * d[nz] / n
    out[nz] = (1.0 - np.exp(-arg)) / arg
    return out


def corr_exponential(d, n_taps: int, tau_rms: float, n_fft: int) -> np.ndarray:
    """r(d) = E{H(k+d) H(k)^*} for taps at delays 0..n_taps-1 with p_l ~ exp(-l/tau_rms).

    The channel law of the Sec. III-A text under Eq. 16 (exponential power-delay
    profile), with integer delays as in Table III.
    """
    d = np.asarray(d, dtype=np.float64)
    l = np.arange(n_taps, dtype=np.float64)
    p = np.exp(-l / tau_rms)
    p = p / p.sum()
    return np.sum(p[:, None] * np.exp(-2j * np.pi * np.outer(l, d.ravel()) / n_fft),
                  axis=0).reshape(d.shape)


def corr_matrix(k_rows, k_cols, r) -> np.ndarray:
    """R[a][b] = r(k_rows[a] - k_cols[b]) (Eq. 16: entries depend on k_a - k_b only).

    The index convention is the one the worked 3W example prints (Eq. W1-W3, P):
    row a is the estimated subcarrier, column b the LS subcarrier.
    """
    ka = np.asarray(k_rows, dtype=np.float64)[:, None]
    kb = np.asarray(k_cols, dtype=np.float64)[None, :]
    return r(ka - kb)


def lmmse_weight(R_h_hls: np.ndarray, R_hh: np.ndarray, sigma2: float) -> np.ndarray:
    """Eq. 13 / 17: W = R_{H Hls} (R_{HH} + sigma2 / sigma_s^2 I)^-1, sigma_s^2 = 1.

    Right division by LU with partial pivoting: W A = R  <=>  A^T W^T = R^T.
    """
    A = R_hh + sigma2 * np.eye(R_hh.shape[0])
    return np.linalg.solve(A.T, R_h_hls.T).T


def subblock_weights(n_sc: int, B: int, r, sigma2: float) -> list:
    """One (start, W) per non-overlapping block of B contiguous subcarriers.

    Per block: R = [r(k_a - k_b)] over its own subcarriers, W = R (R + sigma2 I)^-1.
    """
    out = []
    for b0 in range(0, n_sc, B):
        idx = np.arange(b0, min(b0 + B, n_sc))
        R = corr_matrix(idx, idx, r)
        out.append((b0, lmmse_weight(R, R, sigma2)))
    return out


def subblock_lmmse(h_ls: np.ndarray, B: int, r, sigma2: float, weights=None) -> np.ndarray:
    """Eq. 12 per block: H_LMMSE[blk] = W_blk H_LS[blk] for every (slot, user, antenna).

    ``weights`` (optional) replaces the model weights: a list of (start, W).
    """
    h_ls = np.asarray(h_ls, dtype=np.complex128)
    n_sc = h_ls.shape[-1]
    if weights is None:
        weights = subblock_weights(n_sc, B, r, sigma2)
    out = np.empty_like(h_ls)
    for b0, W in weights:
        n = W.shape[0]
        blk = h_ls[..., b0:b0 + n]                   # [...][n]
        out[..., b0:b0 + n] = blk @ W.T               # row-wise W @ h
    return out


# ------------------------------------------------------------ MMSE detection
def mmse_detect(h: np.ndarray, y_data: np.ndarray, sigma2: float, n_data_per_slot: int):
    """Eq. 20-22 per (slot, subcarrier): (H^H H + sigma2 I) x~ = H^H y, solved by LU.

    h [T][K][M][N], y_data [T*D][M][N].  Returns
      x_eq [T*D][K][N]   the MMSE output x~ of Eq. 22
      s    [T][K][N]     sigma2 [A^-1]_kk (so mu = 1 - s, nu = s / (1 - s))
    """
    h = np.asarray(h, dtype=np.complex128)
    y = np.asarray(y_data, dtype=np.complex128)
    T, K, M, N = h.shape
    D = n_data_per_slot
    x_eq = np.empty((T * D, K, N), dtype=np.complex128)
    s = np.empty((T, K, N), dtype=np.float64)
    for t in range(T):
        Hk = np.transpose(h[t], (2, 1, 0))                     # [N][M][K]
        HkH = np.conj(np.transpose(Hk, (0, 2, 1)))            # [N][K][M]
        A = HkH @ Hk + sigma2 * np.eye(K)                      # Eq. 22 left side
        Yk = np.transpose(y[t * D:(t + 1) * D], (2, 1, 0))    # [N][M][D]
        Z = HkH @ Yk                                           # Eq. 22 right side
        X = np.linalg.solve(A, Z)                              # [N][K][D]
        x_eq[t * D:(t + 1) * D] = np.transpose(X, (2, 1, 0))
        Ainv = np.linalg.inv(A)
        s[t] = (sigma2 * np.real(np.diagonal(Ainv, axis1=1, axis2=2))).T
    return x_eq, s


def gram_matched_filter(h: np.ndarray, y_data: np.ndarray, sigma2: float, n_data_per_slot: int):
    """The two sides of Eq. 22 per (slot, subcarrier): A = H^H H + sigma2 I and z = H^H y.

    h [T][K][M][N], y_data [T*D][M][N].  Returns A [T][N][K][K] and z [T][N][K][D].
    """
    h = np.asarray(h, dtype=np.complex128)
    y = np.asarray(y_data, dtype=np.complex128)
    T, K, M, N = h.shape
    D = n_data_per_slot
    A = np.empty((T, N, K, K), dtype=np.complex128)
    z = np.empty((T, N, K, D), dtype=np.complex128)
    for t in range(T):
        Hk = np.transpose(h[t], (2, 1, 0))                     # [N][M][K]
        HkH = np.conj(np.transpose(Hk, (0, 2, 1)))            # [N][K][M]
        A[t] = HkH @ Hk + sigma2 * np.eye(K)
        z[t] = HkH @ np.transpose(y[t * D:(t + 1) * D], (2, 1, 0))
    return A, z


def round_half(x: np.ndarray, fmt: str) -> np.ndarray:
    """Round every real and imaginary part to a 16-bit float, nearest, ties to even:
    fmt "bf16" (8 significant bits, FP32 exponent range) or "fp16" (IEEE binary16).
    Used to model the operands a 16-bit product consumes; values stay float64."""
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return round_half(x.real, fmt) + 1j * round_half(x.imag, fmt)
    if fmt == "fp16":
        return x.astype(np.float32).astype(np.float16).astype(np.float64)
    # bf16: keep the top 16 bits of the FP32 pattern, rounding the dropped 16 to nearest even
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def refined_mmse_detect(h: np.ndarray, y_data: np.ndarray, sigma2: float, n_data_per_slot: int,
                        A_low: np.ndarray, z_low: np.ndarray):
    """One step of iterative refinement of Eq. 22 around an approximate system.

    The solve uses the approximate Gram A_low and right side z_low ([T][N][K][K], [T][N][K][D]):
      x0 = A_low^-1 z_low,
      r  = H^H (y - H x0) - sigma2 x0      (the residual of Eq. 22 from the given H),
      x1 = x0 + A_low^-1 r.
    Returns x1 [T*D][K][N] and s = sigma2 [A_low^-1]_kk [T][K][N].
    """
    h = np.asarray(h, dtype=np.complex128)
    y = np.asarray(y_data, dtype=np.complex128)
    T, K, M, N = h.shape
    D = n_data_per_slot
    x1 = np.empty((T * D, K, N), dtype=np.complex128)
    s = np.empty((T, K, N), dtype=np.float64)
    for t in range(T):
        Hk = np.transpose(h[t], (2, 1, 0))                     # [N][M][K]
        HkH = np.conj(np.transpose(Hk, (0, 2, 1)))            # [N][K][M]
        Yk = np.transpose(y[t * D:(t + 1) * D], (2, 1, 0))    # [N][M][D]
        x0 = np.linalg.solve(A_low[t], z_low[t])               # [N][K][D]
        r = HkH @ (Yk - Hk @ x0) - sigma2 * x0
        x = x0 + np.linalg.solve(A_low[t], r)
        x1[t * D:(t + 1) * D] = np.transpose(x, (2, 1, 0))
        s[t] = (sigma2 * np.real(np.diagonal(np.linalg.inv(A_low[t]), axis1=1, axis2=2))).T
    return x1, s


def zf_detect(h: np.ndarray, y_data: np.ndarray, n_data_per_slot: int) -> np.ndarray:
    """Eq. 18-19: x~ = (H^H H)^-1 H^H y per (slot, subcarrier), by LU."""
    x, _ = mmse_detect(h, y_data, 0.0, n_data_per_slot)
    return x


# ------------------------------------------------------------------- demapper
def _gray_to_binary(g: int) -> int:
    b = 0
    while g:
        b ^= g
        g >>= 1
    return b


def constellation(q: int) -> np.ndarray:
    """Gray QAM table indexed by label (b0 = MSB): even bits on I, odd bits on Q.

    Per dimension with m = q/2 bits read MSB first: level = (2^m - 1) - 2 gray^-1(bits),
    so bit value 0 of the leading bit is the positive half; unit mean energy.
    """
    m = q // 2
    pts = np.empty(1 << q, dtype=np.complex128)
    for label in range(1 << q):
        bits = [(label >> (q - 1 - i)) & 1 for i in range(q)]

        def level(bs):
            g = 0
            for b in bs:
                g = (g << 1) | b
            return ((1 << m) - 1) - 2 * _gray_to_binary(g)

        pts[label] = level(bits[0::2]) + 1j * level(bits[1::2])
    return pts / np.sqrt(2.0 * (4 ** m - 1) / 3.0)


def unbias(x_eq: np.ndarray, s: np.ndarray, n_data_per_slot: int):
    """x^ = x~ / mu and nu = (1 - mu) / mu with mu = 1 - s, per data symbol."""
    D = n_data_per_slot
    s_d = np.repeat(s, D, axis=0)                 # [T*D][K][N]
    mu = 1.0 - s_d
    return x_eq / mu, s_d / mu


def hard_decision(xhat: np.ndarray, q: int) -> np.ndarray:
    """Nearest constellation point (argmin over the whole table), as its label."""
    pts = constellation(q)
    d2 = np.abs(xhat[..., None] - pts) ** 2
    return np.argmin(d2, axis=-1).astype(np.int64)


def maxlog_llr(xhat: np.ndarray, nu: np.ndarray, q: int) -> np.ndarray:
    """Max-log LLR per bit: (min_{b_i=1} |x^-x|^2 - min_{b_i=0} |x^-x|^2) / nu; > 0 favours 0."""
    pts = constellation(q)
    labels = np.arange(1 << q)
    d2 = np.abs(xhat[..., None] - pts) ** 2
    out = np.empty(xhat.shape + (q,), dtype=np.float64)
    for i in range(q):
        bit = (labels >> (q - 1 - i)) & 1
        out[..., i] = (d2[..., bit == 1].min(axis=-1) - d2[..., bit == 0].min(axis=-1)) / nu
    return out


def boundary_margin(xhat: np.ndarray, q: int) -> np.ndarray:
    """Distance of x^ to the nearest per-dimension decision boundary, in units of d_min/2.

    Boundaries of the Gray PAM slicer sit halfway between adjacent levels (and the
    decision is per dimension because the table is a product of two PAM sets).
    """
    m = q // 2
    scale = np.sqrt(2.0 * (4 ** m - 1) / 3.0)
    bounds = np.arange(-(1 << m) + 2, (1 << m) - 1, 2, dtype=np.float64)  # between levels
    if bounds.size == 0:
        return np.full(xhat.shape, np.inf)
    dist = []
    for comp in (np.real(xhat) * scale, np.imag(xhat) * scale):
        dist.append(np.min(np.abs(comp[..., None] - bounds), axis=-1))
    return np.minimum(dist[0], dist[1])


# ------------------------------------------------- comb pilots (Sec. II, IV-B)
# The paper's deployed pilot structure: the pilot OFDM symbol is shared by the users on
# disjoint tones, user k (0-based) on subcarriers k, k + S, k + 2S, ... (Sec. II, Fig. 1;
# S = 12 there).  Layouts: y_pilot [T][M][N_sc], pilots [T][N_sc] (the value sent on each
# tone by its owner), h_ls [T][K][M][P] on the P = N_sc / S tones of each user.
COMB_3W, COMB_SW, COMB_INTERP3 = "3W", "SW", "interp3"


def comb_tones(k: int, S: int, n_sc: int) -> np.ndarray:
    """Pilot subcarriers of user k: k, k + S, ... < n_sc (Sec. II)."""
    return np.arange(k, n_sc, S)


def comb_ls(y_pilot: np.ndarray, pilots: np.ndarray, K: int, S: int) -> np.ndarray:
    """Eq. 9 on each user's own tones: h_ls[t][k][m][i] = y_p[t][m][k + iS] / p[t][k + iS]."""
    y_pilot = np.asarray(y_pilot, dtype=np.complex128)
    pilots = np.asarray(pilots, dtype=np.complex128)
    n_sc = y_pilot.shape[-1]
    out = []
    for k in range(K):
        tn = comb_tones(k, S, n_sc)
        out.append(y_pilot[:, :, tn] / pilots[:, None, tn])
    return np.stack(out, axis=1)


def comb_groups(method: str, k: int, S: int, n_sc: int) -> list:
    """Group map of Table I (3W) and Table II (S-W, 12W at S = 12) for user k, 0-based.

    One group per pilot index j = 0..P-1, each a list of estimated subcarriers, the first
    of the Q consecutive LS tones it uses (window i0) and the index of its weight matrix:
      3W:  Q = 3, estimates at the user's tone j and S/3, 2S/3 after it;
      S-W: Q = S, estimates at the S subcarriers jS .. jS + S - 1 (the same for all users);
      window i0 = min(max(j - (Q - 1) // 2, 0), P - Q), weight index j - i0 (edge groups
      get their own W, all interior groups share one, Sec. IV-B).
    """
    P = len(comb_tones(k, S, n_sc))
    Q = 3 if method == COMB_3W else S
    half = (Q - 1) // 2
    groups = []
    for j in range(P):
        i0 = min(max(j - half, 0), P - Q)
        if method == COMB_3W:
            out = k + j * S + np.arange(3) * (S // 3)
        else:
            out = j * S + np.arange(S)
        groups.append((out, i0, j - i0))
    return groups


def comb_weight(out_sc, in_sc, r, sigma2: float) -> np.ndarray:
    """Eq. 17 with a rectangular cross-correlation (Eq. W1-W3, P):
    W = R_{H Hls} (R_{Hls Hls} + sigma2 I)^-1, R_{H Hls}[a][b] = r(out_a - in_b),
    R_{Hls Hls}[a][b] = r(in_a - in_b)."""
    return lmmse_weight(corr_matrix(out_sc, in_sc, r), corr_matrix(in_sc, in_sc, r), sigma2)


def zero_order_hold(pos: np.ndarray, vals: np.ndarray, n_sc: int) -> np.ndarray:
    """Every subcarrier n takes the estimate at the last position <= n (Sec. IV-C, on the
    detector's input); subcarriers before the first position take the first estimate."""
    order = np.argsort(pos, kind="stable")
    pos, vals = np.asarray(pos)[order], vals[..., order]
    idx = np.searchsorted(pos, np.arange(n_sc), side="right") - 1
    return vals[..., np.maximum(idx, 0)]


def comb_lmmse(h_ls: np.ndarray, method: str, S: int, n_sc: int, r, sigma2: float) -> np.ndarray:
    """3W- / S-W-LMMSE (Sec. IV-B): per group, W (Q estimates x Q LS tones) times the
    group's LS window (Eq. 12); 3W estimates are then held to every subcarrier.
    Returns h [T][K][M][n_sc]."""
    h_ls = np.asarray(h_ls, dtype=np.complex128)
    T, K, M, _ = h_ls.shape
    out = np.empty((T, K, M, n_sc), dtype=np.complex128)
    for k in range(K):
        tones = comb_tones(k, S, n_sc)
        pos, vals = [], []
        for o, i0, _ in comb_groups(method, k, S, n_sc):
            Q = 3 if method == COMB_3W else S
            W = comb_weight(o, tones[i0:i0 + Q], r, sigma2)
            pos.append(o)
            vals.append(h_ls[:, k, :, i0:i0 + Q] @ W.T)
        pos = np.concatenate(pos)
        vals = np.concatenate(vals, axis=-1)
        if method == COMB_3W:
            out[:, k] = zero_order_hold(pos, vals, n_sc)
        else:
            keep = pos < n_sc
            out[:, k][..., pos[keep]] = vals[..., keep]
    return out


def comb_interp3_ls(h_ls: np.ndarray, S: int, n_sc: int) -> np.ndarray:
    """Three-fold linearly interpolated LS (Sec. III-A, the comparator of Sec. V): at the
    3W positions k + jS + uS/3 the LS of tones j and j+1 weighted (1 - u/3, u/3); past the
    last tone its LS is held; then zero-order hold to every subcarrier."""
    h_ls = np.asarray(h_ls, dtype=np.complex128)
    T, K, M, P = h_ls.shape
    out = np.empty((T, K, M, n_sc), dtype=np.complex128)
    for k in range(K):
        pos, vals = [], []
        for j in range(P):
            for u in range(3):
                pos.append(k + j * S + u * (S // 3))
                if j + 1 < P:
                    vals.append((1 - u / 3) * h_ls[:, k, :, j] + (u / 3) * h_ls[:, k, :, j + 1])
                else:
                    vals.append(h_ls[:, k, :, j])
        out[:, k] = zero_order_hold(np.array(pos), np.stack(vals, axis=-1), n_sc)
    return out


def comb_receive_subframe(y_pilot, pilots, y_data, *, K: int, S: int, method: str, sigma2: float, r,
                          n_data_per_slot: int, q: int) -> dict:
    """Comb-pilot LS -> 3W / S-W LMMSE or interpolated LS -> MMSE detection -> demap."""
    n_sc = np.asarray(y_pilot).shape[-1]
    h_ls = comb_ls(y_pilot, pilots, K, S)
    if method == COMB_INTERP3:
        h = comb_interp3_ls(h_ls, S, n_sc)
    else:
        h = comb_lmmse(h_ls, method, S, n_sc, r, sigma2)
    x_eq, s = mmse_detect(h, y_data, sigma2, n_data_per_slot)
    xhat, nu = unbias(x_eq, s, n_data_per_slot)
    return dict(h_ls=h_ls, h=h, x_eq=x_eq, s=s, xhat=xhat, nu=nu,
                labels=hard_decision(xhat, q), llr=maxlog_llr(xhat, nu, q))


# ---------------------------------------------------------------- whole path
def receive_subframe(y_pilot, pilots, y_data, *, B: int, sigma2: float, r,
                     n_data_per_slot: int, q: int, weights=None) -> dict:
    """LS (Eq. 9) -> sub-block LMMSE (Eq. 12, 17) -> MMSE detection (Eq. 22) -> demap."""
    h_ls = ls_estimate(y_pilot, pilots)
    h = subblock_lmmse(h_ls, B, r, sigma2, weights)
    x_eq, s = mmse_detect(h, y_data, sigma2, n_data_per_slot)
    xhat, nu = unbias(x_eq, s, n_data_per_slot)
    return dict(h_ls=h_ls, h=h, x_eq=x_eq, s=s, xhat=xhat, nu=nu,
                labels=hard_decision(xhat, q), llr=maxlog_llr(xhat, nu, q))


def make_r(pdp: str, *, n_taps=None, tau_rms=None, n_fft=None, L=None, n=None):
    """The correlation function r(d) for a PDP kind ('exp' or 'uniform_L')."""
    if pdp == "exp":
        return lambda d: corr_exponential(d, n_taps, tau_rms, n_fft)
    if pdp == "uniform_L":
        return lambda d: corr_uniform_L(d, L, n)
    raise ValueError(pdp)
