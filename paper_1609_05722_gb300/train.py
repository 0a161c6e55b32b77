"""Prior training through the unrolled solve: a torch.autograd.Function over foe_train_step.

loss = FoEUnrolledLoss.apply(filters, log_alpha, clean, noisy, iters, lam, gamma, tau, ckpt_every)

filters (nf, 7, 7) and log_alpha (nf,) are the parameters (weights alpha_i = exp(log_alpha_i), Eq.
learningmodel); clean and noisy are CUDA tensors of shape (B, H, ld) holding H x W images.  The loss is
sum_s 1/2 ||I_C(u_s^T) - g_s||^2 after `iters` iPiano steps of the Anscombe quadratic model.  The
forward pass runs the CUDA training step once, which returns the loss and both gradients; backward
scales the stored gradients.  tau is a constant of the solve (no gradient flows into it).
"""
from __future__ import annotations

import os

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


class FoEImplicitLoss(torch.autograd.Function):
    """The same objective with the paper's own gradient: implicit differentiation at u^T (Sec. 2.5, Eq.
    implicitdifferentiation and Eq. overallderivative), q = H_E(u^T)^{-1} dL/dw by conjugate gradients on the device.

    loss = FoEImplicitLoss.apply(filters, log_alpha, clean, noisy, iters, lam, gamma, tau, max_cg, cg_tol)

    Exact at a minimiser of the lower-level problem, so `iters` should let the solve converge; tau = 0 takes the
    certified step of the current filters (the gradient does not depend on tau once u^T is the minimiser)."""

    @staticmethod
    def forward(ctx, filters, log_alpha, clean, noisy, iters: int, lam: float, gamma: float, tau: float,
                max_cg: int = 200, cg_tol: float = 1e-5, W: int | None = None):
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
            loss, _ = F.foe_train_grad_implicit(handle, clean, noisy, B, H, W, ld, opts, dk, dla, int(max_cg),
                                                float(cg_tol))
        finally:
            F.foe_destroy(handle)
        ctx.save_for_backward(dk.view(-1, 7, 7).to(filters.device, filters.dtype), dla.to(log_alpha.device, log_alpha.dtype))
        return torch.tensor(loss, dtype=torch.float64, device=filters.device)

    @staticmethod
    def backward(ctx, grad_out):
        dk, dla = ctx.saved_tensors
        g = grad_out.to(dk.dtype)
        return g * dk, g * dla, None, None, None, None, None, None, None, None, None


class DataParallelLoss(torch.autograd.Function):
    """Data-parallel training over ranks that each hold a share of the training pairs (the loss of Sec. 3.2 is a
    sum over samples, so the batch splits freely).

    loss = DataParallelLoss.apply(filters, log_alpha, local_loss_fn, dist)

    local_loss_fn(filters, log_alpha) is this rank's loss (for instance FoEUnrolledLoss or FoEImplicitLoss over its
    images).  The forward pass evaluates it and its gradients, then sums the loss and the gradients (nf x 49 filter
    coefficients and nf log-weights) over the ranks with one all-reduce of one FP64 vector; every rank returns the
    whole batch's loss, and backward gives the whole batch's gradients, so ranks that start from the same
    parameters take the same optimizer steps (lbfgs_train runs unchanged on every rank)."""

    @staticmethod
    def forward(ctx, filters, log_alpha, local_loss_fn, dist, group=None):
        with torch.enable_grad():
            k = filters.detach().requires_grad_(True)
            la = log_alpha.detach().requires_grad_(True)
            local = local_loss_fn(k, la)
            gk, gla = torch.autograd.grad(local, (k, la))
        # NCCL reduces device tensors, gloo host tensors
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
        v = torch.cat([local.detach().reshape(1).double().to(dev), gk.detach().reshape(-1).double().to(dev),
                       gla.detach().reshape(-1).double().to(dev)])
        dist.all_reduce(v, group=group)
        nk = gk.numel()
        ctx.save_for_backward(v[1:1 + nk].view_as(gk).to(filters.device, filters.dtype),
                              v[1 + nk:].view_as(gla).to(log_alpha.device, log_alpha.dtype))
        return v[0].to(device=filters.device)

    @staticmethod
    def backward(ctx, grad_out):
        gk, gla = ctx.saved_tensors
        return grad_out.to(gk.dtype) * gk, grad_out.to(gla.dtype) * gla, None, None, None


def lbfgs_train(loss_fn, filters, log_alpha, max_iter: int = 500, tol: float = 1e-5, history: int = 10,
                on_step=None, checkpoint: str | None = None):
    """Algorithm 1 (Sec. 2.5): L-BFGS over the filters and log-weights of the prior.

    loss_fn(filters, log_alpha) returns the training loss as a differentiable scalar tensor (for instance
    FoEImplicitLoss.apply or FoEUnrolledLoss.apply with the data bound).  Each iteration is one L-BFGS step with a
    strong-Wolfe line search; training stops when the relative change of the loss falls below tol, after max_iter
    iterations, or when a step fails to decrease the loss (the three criteria of the paper's training).
    on_step(iteration, loss), if given, is called after every step.  Returns (filters, log_alpha, losses, reason),
    losses[0] being the initial loss.

    checkpoint, if given, is a file path: after every step the training state (parameters, the L-BFGS history and
    line-search state, the losses so far) is written there (atomically, with torch.save), and a call that finds the
    file resumes from it, the filters / log_alpha arguments then serving only as templates; max_iter counts the
    steps of the whole run.  A resumed run takes the same steps as an uninterrupted one.  The stopping decision of
    a step is taken before its checkpoint is written and is stored in it, so a run resumed from the checkpoint of a
    run that had already stopped returns at once with the stored result; a checkpoint without a stored decision has
    the criteria re-checked on its last two losses."""
    k = filters.detach().clone().requires_grad_(True)
    la = log_alpha.detach().clone().requires_grad_(True)
    # one L-BFGS iteration per step; the line search may take up to 20 evaluations within it
    opt = torch.optim.LBFGS([k, la], lr=1.0, max_iter=1, max_eval=20, history_size=history,
                            line_search_fn="strong_wolfe")

    def closure():
        opt.zero_grad()
        L = loss_fn(k, la)
        L.backward()
        return L

    start = 0
    if checkpoint is not None and os.path.exists(checkpoint):
        st = torch.load(checkpoint, weights_only=False)
        with torch.no_grad():
            k.copy_(st["filters"])
            la.copy_(st["log_alpha"])
        opt.load_state_dict(st["optimizer"])
        losses, start = list(st["losses"]), int(st["iteration"])
        stopped = st.get("reason")
        if stopped is None and len(losses) >= 2:
            stopped = _stop_reason(losses[-2], losses[-1], tol)
        if stopped is not None:
            return k.detach(), la.detach(), losses, stopped
    else:
        with torch.no_grad():
            losses = [float(loss_fn(k, la))]
    reason = "max_iter"
    for it in range(start, max_iter):
        opt.step(closure)
        with torch.no_grad():
            L = float(loss_fn(k, la))
        prev = losses[-1]
        losses.append(L)
        stop = _stop_reason(prev, L, tol)
        if checkpoint is not None:
            tmp = f"{checkpoint}.tmp{os.getpid()}"
            torch.save({"filters": k.detach().clone(), "log_alpha": la.detach().clone(),
                        "optimizer": opt.state_dict(), "losses": losses, "iteration": it + 1, "reason": stop}, tmp)
            os.replace(tmp, checkpoint)
        if on_step is not None:
            on_step(it + 1, L)
        if stop is not None:
            reason = stop
            break
    return k.detach(), la.detach(), losses, reason


def _stop_reason(prev: float, L: float, tol: float):
    """The stopping rules of the training loop after a step from loss prev to loss L: a step that does not decrease
    the loss, or a relative change of at most tol; None to go on."""
    if not L < prev:
        return "no_decrease"
    if abs(prev - L) <= tol * abs(prev):
        return "tol"
    return None
