"""Differentiable FP64 oracle of the receive path's symbol MSE (LS -> sub-block LMMSE -> MMSE).

TEST INFRASTRUCTURE, like ``rapro_oracle``: only the tests, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU legs may import it; it shares no code with the CUDA library.

The forward pass restates Eq. 9, 12, 13/17 (with the exponential power-delay profile of
Sec. III-A on integer taps) and 22 in plain PyTorch CPU ops on float64 / complex128, and
torch.autograd supplies the gradient; nothing here is a hand-written adjoint.  The loss is
the mean squared error of the MMSE output against known transmitted symbols,
  L = mean_{data symbol, user, subcarrier} |x~ - x|^2,
as a function of the estimator's noise variance and PDP decay constant (sigma2_est, tau)
and of the detector's noise variance sigma2_det (the receiver uses one sigma2 for both;
keeping them apart lets each path of the gradient be checked).

Layouts as in the C ABI: y_pilot [T][K][M][N], pilots [T][K][N], y_data [T*D][M][N],
x [T*D][K][N].
"""
from __future__ import annotations

import numpy as np
import torch

F64, C128 = torch.float64, torch.complex128


def corr_exp(d: torch.Tensor, n_taps: int, tau: torch.Tensor, n_fft: int) -> torch.Tensor:
    """r(d) = sum_l p_l exp(-j 2 pi l d / n_fft), p_l = exp(-l / tau) / sum_m exp(-m / tau)."""
    l = torch.arange(n_taps, dtype=F64)
    p = torch.exp(-l / tau)
    p = p / p.sum()
    ph = torch.exp(-2j * np.pi * torch.outer(l, d.to(F64)) / n_fft)          # [n_taps][len(d)]
    return p.to(C128) @ ph


def block_weight(n: int, sigma2: torch.Tensor, tau: torch.Tensor, n_taps: int, n_fft: int) -> torch.Tensor:
    """Eq. 13/17 on one block of n subcarriers: W = R (R + sigma2 I)^-1, R[a][b] = r(a - b)."""
    idx = torch.arange(n)
    R = corr_exp((idx[:, None] - idx[None, :]).reshape(-1), n_taps, tau, n_fft).reshape(n, n)
    A = R + sigma2.to(C128) * torch.eye(n, dtype=C128)
    return torch.linalg.solve(A.T, R.T).T                                     # right division


def symbol_mse(y_pilot, pilots, y_data, x, *, B: int, n_taps: int, n_fft: int, n_data_per_slot: int,
               sigma2_est: torch.Tensor, tau: torch.Tensor, sigma2_det: torch.Tensor,
               weights=None):
    """L(sigma2_est, tau, sigma2_det) and the MMSE output x~ [T*D][K][N].

    ``weights`` (optional) replaces the model weights by given tensors (main, tail), so that
    the gradient with respect to W itself can be taken.
    """
    yp = torch.as_tensor(np.asarray(y_pilot), dtype=C128)
    p = torch.as_tensor(np.asarray(pilots), dtype=C128)
    yd = torch.as_tensor(np.asarray(y_data), dtype=C128)
    xt = torch.as_tensor(np.asarray(x), dtype=C128)
    T, K, M, N = yp.shape
    D = n_data_per_slot
    h_ls = yp * torch.conj(p)[:, :, None, :] / (torch.abs(p) ** 2)[:, :, None, :]   # Eq. 9
    tail = N % B
    if weights is None:
        Wm = block_weight(B, sigma2_est, tau, n_taps, n_fft)
        Wt = block_weight(tail, sigma2_est, tau, n_taps, n_fft) if tail else None
    else:
        Wm, Wt = weights
    parts = []
    for b0 in range(0, N, B):                                                 # Eq. 12 per block
        n = min(B, N - b0)
        W = Wm if n == B else Wt
        parts.append(h_ls[..., b0:b0 + n] @ W.T)
    h = torch.cat(parts, dim=-1)                                              # [T][K][M][N]
    xs = []
    for t in range(T):
        Hn = h[t].permute(2, 1, 0)                                            # [N][M][K]
        HnH = torch.conj(Hn.transpose(1, 2))
        A = HnH @ Hn + sigma2_det.to(C128) * torch.eye(K, dtype=C128)        # Eq. 22
        Z = HnH @ yd[t * D:(t + 1) * D].permute(2, 1, 0)                      # [N][K][D]
        xs.append(torch.linalg.solve(A, Z).permute(2, 1, 0))                  # [D][K][N]
    x_eq = torch.cat(xs, dim=0)
    loss = torch.mean(torch.abs(x_eq - xt) ** 2)
    return loss, x_eq


def grads(y_pilot, pilots, y_data, x, *, B, n_taps, n_fft, n_data_per_slot, sigma2_est, tau, sigma2_det):
    """L and dL/d(sigma2_est, tau, sigma2_det) by torch.autograd, as Python floats."""
    s_e = torch.tensor(float(sigma2_est), dtype=F64, requires_grad=True)
    ta = torch.tensor(float(tau), dtype=F64, requires_grad=True)
    s_d = torch.tensor(float(sigma2_det), dtype=F64, requires_grad=True)
    loss, _ = symbol_mse(y_pilot, pilots, y_data, x, B=B, n_taps=n_taps, n_fft=n_fft,
                         n_data_per_slot=n_data_per_slot, sigma2_est=s_e, tau=ta, sigma2_det=s_d)
    loss.backward()
    return float(loss.detach()), float(s_e.grad), float(ta.grad), float(s_d.grad)


def weight_grads(y_pilot, pilots, y_data, x, *, B, n_taps, n_fft, n_data_per_slot, sigma2_est, tau,
                 sigma2_det):
    """dL/dW* for the main and tail weights (the conjugate Wirtinger gradient, so that
    dL = 2 Re sum conj(G) dW), and dL/dsigma2_det with W held fixed."""
    s_e = torch.tensor(float(sigma2_est), dtype=F64)
    ta = torch.tensor(float(tau), dtype=F64)
    N = np.asarray(y_pilot).shape[-1]
    tail = N % B
    Wm = block_weight(B, s_e, ta, n_taps, n_fft).detach().requires_grad_(True)
    Wt = block_weight(tail, s_e, ta, n_taps, n_fft).detach().requires_grad_(True) if tail else None
    s_d = torch.tensor(float(sigma2_det), dtype=F64, requires_grad=True)
    loss, _ = symbol_mse(y_pilot, pilots, y_data, x, B=B, n_taps=n_taps, n_fft=n_fft,
                         n_data_per_slot=n_data_per_slot, sigma2_est=s_e, tau=ta, sigma2_det=s_d,
                         weights=(Wm, Wt))
    loss.backward()
    # torch's .grad of a real loss with respect to a complex leaf is 2 dL/dW* (for L = |z|^2
    # it is 2 z), so G = grad / 2.
    g_m = Wm.grad.numpy() / 2.0
    g_t = Wt.grad.numpy() / 2.0 if tail else None
    return float(loss.detach()), g_m, g_t, float(s_d.grad)
