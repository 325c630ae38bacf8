"""Differentiable receive: torch.autograd over the library's forward and adjoint kernels.

``symbol_mse(theta, batch, shape)`` returns the mean squared error of the MMSE output
against known transmitted symbols, averaged over a batch of subframes, as a function of
theta = (sigma2, tau_rms) -- the noise variance used by the estimator (Eq. 17) and the
detector (Eq. 22), and the decay constant of the exponential PDP model behind R_b.  Its
gradient comes from ``rapro_mse_backward`` (the detector's adjoint and the weight gradient,
CUDA) and ``rapro_weight_grad_host`` (the FP64 chain rule through W = R (R + sigma2 I)^-1).
``symbol_mse_weights(w_main, w_tail, sigma2, batch, shape)`` makes the block weights of
Eq. 12 themselves the parameters (tied over the full blocks, the tail block's own), with
the detector's sigma2: the forward filters with them through the library's weight
override, and the backward returns torch's gradient 2 dL/dW* from the same
``rapro_mse_backward`` call.
This module only marshals arguments and sums the per-subframe results.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rapro as R


class _SymbolMSE(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, batch, shape):
        sigma2, tau = float(theta[0]), float(theta[1])
        p = R.make_params(**shape, sigma2=sigma2, tau_rms=tau)
        plan = R.Plan(p)
        s = plan.shapes()
        dev = batch[0]["y_pilot"].device
        c64 = torch.complex64
        h = torch.empty(s["h"], dtype=c64, device=dev)
        g_h = torch.empty(s["h"], dtype=c64, device=dev)
        x = torch.empty(s["x_eq"], dtype=c64, device=dev)
        scal = torch.empty(2, dtype=torch.float32, device=dev)
        B, tail = p.subblock, plan.tail
        gwm = torch.empty((B, B), dtype=c64, device=dev)
        gwt = torch.empty((tail, tail), dtype=c64, device=dev) if tail else None
        loss = g_sd = 0.0
        G_m = np.zeros((B, B), np.complex128)
        G_t = np.zeros((tail, tail), np.complex128) if tail else None
        for d in batch:
            R.rapro_receive_subframe(plan, d["y_pilot"], d["pilots"], d["y_data"], x, h_out=h)
            R.rapro_mse_backward(plan, d["y_pilot"], d["pilots"], d["y_data"], h, x, d["x_ref"], g_h, scal, gwm, gwt)
            sc = scal.cpu().double().numpy()
            loss += sc[0]
            g_sd += sc[1]
            G_m += gwm.cpu().numpy()
            if tail:
                G_t += gwt.cpu().numpy()
        if plan.device_status() != 0:
            raise RuntimeError("a receive kernel reported a pipeline timeout")
        n = len(batch)
        g_s2_w, g_tau = R.rapro_weight_grad_host(p, G_m, G_t)
        plan.close()
        ctx.grad = torch.tensor([(g_sd + g_s2_w) / n, g_tau / n], dtype=torch.float64)
        return torch.tensor(loss / n, dtype=torch.float64)

    @staticmethod
    def backward(ctx, g_out):
        return g_out * ctx.grad, None, None


class _SymbolMSEWeights(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w_main, w_tail, sigma2, batch, shape):
        p = R.make_params(**shape, sigma2=float(sigma2))
        plan = R.Plan(p)
        s = plan.shapes()
        dev = batch[0]["y_pilot"].device
        c64 = torch.complex64
        B, tail, nb = p.subblock, plan.tail, plan.nb
        n_full = nb - (1 if tail else 0)
        parts = [w_main.detach().to(dev, c64).reshape(-1)] * n_full
        if tail:
            parts.append(w_tail.detach().to(dev, c64).reshape(-1))
        w_over = torch.cat(parts).contiguous()                 # one W per block, as rapro.h lays out
        h = torch.empty(s["h"], dtype=c64, device=dev)
        g_h = torch.empty(s["h"], dtype=c64, device=dev)
        x = torch.empty(s["x_eq"], dtype=c64, device=dev)
        scal = torch.empty(2, dtype=torch.float32, device=dev)
        gwm = torch.empty((B, B), dtype=c64, device=dev)
        gwt = torch.empty((tail, tail), dtype=c64, device=dev) if tail else None
        loss = g_sd = 0.0
        G_m = torch.zeros((B, B), dtype=torch.complex128)
        G_t = torch.zeros((tail, tail), dtype=torch.complex128) if tail else None
        for d in batch:
            R.rapro_ce_ls_lmmse(plan, d["y_pilot"], d["pilots"], h, w_override=w_over)
            R.rapro_mmse_detect(plan, h, d["y_data"], x)
            R.rapro_mse_backward(plan, d["y_pilot"], d["pilots"], d["y_data"], h, x, d["x_ref"], g_h, scal, gwm, gwt)
            sc = scal.cpu().double()
            loss += float(sc[0])
            g_sd += float(sc[1])
            G_m += gwm.cpu().to(torch.complex128)
            if tail:
                G_t += gwt.cpu().to(torch.complex128)
        if plan.device_status() != 0:
            raise RuntimeError("a receive kernel reported a pipeline timeout")
        plan.close()
        n = len(batch)
        # torch's gradient of a real loss with respect to a complex tensor is 2 dL/dW*
        ctx.g = (2.0 * G_m / n, (2.0 * G_t / n) if tail else None, g_sd / n)
        ctx.meta = (w_main.dtype, w_main.device, None if w_tail is None else (w_tail.dtype, w_tail.device))
        return torch.tensor(loss / n, dtype=torch.float64)

    @staticmethod
    def backward(ctx, g_out):
        g_m, g_t, g_s = ctx.g
        (dt_m, dv_m, tmeta) = ctx.meta
        gm = (g_out * g_m).to(dv_m, dt_m)
        gt = None if g_t is None or tmeta is None else (g_out * g_t).to(tmeta[1], tmeta[0])
        return gm, gt, (g_out * g_s).to(torch.float64), None, None


def symbol_mse_weights(w_main: torch.Tensor, w_tail, sigma2, batch: list, shape: dict) -> torch.Tensor:
    """L(W) over ``batch`` with the block weights of Eq. 12 as parameters.

    w_main: complex [B][B] (shared by the full blocks), w_tail: complex [tail][tail] or None
    when B divides n_sc, sigma2: the detector's noise variance (a float64 tensor, so that it
    may be learned too).  shape: the other rapro_params fields as make_params keywords (its
    sigma2 and PDP only build the plan's own weights, which the override replaces).
    """
    s2 = sigma2 if isinstance(sigma2, torch.Tensor) else torch.tensor(float(sigma2), dtype=torch.float64)
    return _SymbolMSEWeights.apply(w_main, w_tail, s2, batch, shape)


def symbol_mse(theta: torch.Tensor, batch: list, shape: dict) -> torch.Tensor:
    """L(theta) over ``batch`` (dicts of device tensors y_pilot, pilots, y_data, x_ref).

    theta: CPU float64 tensor [sigma2, tau_rms].  shape: the other rapro_params fields
    (M, K, n_sc, n_fft, subblock, qam_bits, n_taps, ...) as make_params keywords.
    """
    return _SymbolMSE.apply(theta, batch, shape)
