"""Prior training through the unrolled solve: a torch.autograd.Function over foe_train_step.

loss = FoEUnrolledLoss.apply(filters, log_alpha, clean, noisy, iters, lam, gamma, tau, ckpt_every)

filters (nf, 7, 7) and log_alpha (nf,) are the parameters (weights alpha_i = exp(log_alpha_i), Eq.
learningmodel); clean and noisy are CUDA tensors of shape (B, H, ld) holding H x W images.  The loss is
sum_s 1/2 ||I_C(u_s^T) - g_s||^2 after `iters` iPiano steps of the Anscombe quadratic model.  The
forward pass runs the CUDA training step once, which returns the loss and both gradients; backward
scales the stored gradients.  tau is a constant of the solve (no gradient flows into it).
"""
from __future__ import annotations

import numpy as np
import torch

from . import foe as F


class FoEUnrolledLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, filters, log_alpha, clean, noisy, iters: int, lam: float, gamma: float, tau: float,
                ckpt_every: int = 0, W: int | None = None):
        B, H, ld = clean.shape
        W = W or ld
        k = filters.detach().float().cpu().numpy()
        a = np.exp(log_alpha.detach().double().cpu().numpy()).astype(np.float32)
        handle = F.foe_create(k, a)
        try:
            dk = torch.empty((k.shape[0], 49), dtype=torch.float32, device=clean.device)
            dla = torch.empty((k.shape[0],), dtype=torch.float32, device=clean.device)
            opts = F.SolveOpts(model=F.FOE_MODEL_ANS_L2, prec=F.FOE_PREC_FP32, iters=int(iters), lam=float(lam),
                               gamma=float(gamma), tau=float(tau))
            loss = F.foe_train_step(handle, clean, noisy, B, H, W, ld, opts, dk, dla, ckpt_every)
        finally:
            F.foe_destroy(handle)
        ctx.save_for_backward(dk.view(-1, 7, 7).to(filters.device, filters.dtype), dla.to(log_alpha.device, log_alpha.dtype))
        return torch.tensor(loss, dtype=torch.float64, device=filters.device)

    @staticmethod
    def backward(ctx, grad_out):
        dk, dla = ctx.saved_tensors
        g = grad_out.to(dk.dtype)
        return g * dk, g * dla, None, None, None, None, None, None, None, None
