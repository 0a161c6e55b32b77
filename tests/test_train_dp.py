"""Data-parallel training on CPU ranks (gloo): each rank holds half of the training pairs, DataParallelLoss sums
loss and gradients over the ranks with one all-reduce, and the result equals the oracle's gradient of the whole
batch; L-BFGS (Algorithm 1) then takes identical steps on every rank.  The per-rank loss is the oracle's unrolled
training loss and gradient (reverse mode through the iteration)."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_1609_05722_gb300 import synth, train

B, H, W, T, TAU = 4, 12, 11, 3, 2e-3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    clean = np.stack([synth.clean_image(H, W, 300 + s) * 4.0 for s in range(B)])
    noisy = np.stack([synth.poisson_observation(clean[s] / 4.0, 4.0, 400 + s) for s in range(B)])
    return clean, noisy


class _OracleLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, k, la, clean, noisy):
        pr = O.Problem(k.detach().double().numpy(), np.exp(la.detach().double().numpy()), H, W,
                       model=O.MODEL_ANS_L2, lam=1.0, tau=TAU, gamma=0.8, nthreads=1)
        L, dk, da = pr.train_grad(clean, noisy, T)
        ctx.save_for_backward(torch.from_numpy(dk), torch.from_numpy(da))
        return torch.tensor(L, dtype=torch.float64)

    @staticmethod
    def backward(ctx, g):
        dk, da = ctx.saved_tensors
        return g * dk, g * da, None, None


def _params():
    k, a = synth.filter_bank()
    return torch.from_numpy(k.astype(np.float64)), torch.from_numpy(np.log(a.astype(np.float64)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        clean, noisy = _batch()
        share = slice(rank * B // world, (rank + 1) * B // world)

        def local(k, la):
            return _OracleLoss.apply(k, la, clean[share], noisy[share])

        def loss_dp(k, la):
            return train.DataParallelLoss.apply(k, la, local, dist)

        k, la = _params()
        k.requires_grad_(True)
        la.requires_grad_(True)
        L = loss_dp(k, la)
        L.backward()
        first = (float(L), k.grad.numpy().copy(), la.grad.numpy().copy())
        k2, la2, losses, reason = train.lbfgs_train(loss_dp, k.detach(), la.detach(), max_iter=2)
        q.put((rank, first, k2.numpy(), la2.numpy(), losses))
    finally:
        dist.destroy_process_group()


def test_two_ranks_match_the_whole_batch_and_step_together():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r[0], r[1:]) for r in (q.get(timeout=300) for _ in range(2)))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    clean, noisy = _batch()
    k, la = _params()
    pr = O.Problem(k.numpy(), np.exp(la.numpy()), H, W, model=O.MODEL_ANS_L2, lam=1.0, tau=TAU, gamma=0.8,
                   nthreads=1)
    L, dk, da = pr.train_grad(clean, noisy, T)
    for r in (0, 1):
        (L_r, dk_r, da_r), k2, la2, losses = res[r]
        # the two halves' sums, added in another order than the oracle's loop over the batch
        assert abs(L_r - L) <= 1e-12 * abs(L)
        np.testing.assert_allclose(dk_r, dk, rtol=0, atol=1e-11 * np.abs(dk).max())
        np.testing.assert_allclose(da_r, da, rtol=0, atol=1e-11 * np.abs(da).max())
        assert losses[-1] < losses[0]
    # identical global values give identical optimizer steps on both ranks
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])
    assert res[0][3] == res[1][3]
