"""Differentiable receive: torch.autograd over the library's forward and adjoint kernels.

``symbol_mse(theta, batch, shape)`` returns the mean squared error of the MMSE output
against known transmitted symbols, averaged over a batch of subframes, as a function of
theta = (sigma2, tau_rms) -- the noise variance used by the estimator (Eq. 17) and the
detector (Eq. 22), and the decay constant of the exponential PDP model behind R_b.  Its
gradient comes from ``rapro_mse_backward`` (the detector's adjoint and the weight gradient,
CUDA) and ``rapro_weight_grad_host`` (the FP64 chain rule through W = R (R + sigma2 I)^-1).
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


def symbol_mse(theta: torch.Tensor, batch: list, shape: dict) -> torch.Tensor:
    """L(theta) over ``batch`` (dicts of device tensors y_pilot, pilots, y_data, x_ref).

    theta: CPU float64 tensor [sigma2, tau_rms].  shape: the other rapro_params fields
    (M, K, n_sc, n_fft, subblock, qam_bits, n_taps, ...) as make_params keywords.
    """
    return _SymbolMSE.apply(theta, batch, shape)
