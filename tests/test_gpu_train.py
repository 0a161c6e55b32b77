"""Hand-written backward of the unrolled solve vs the FP64 oracle gradient (itself pinned by central
finite differences in the oracle tests).

FP32 gradients are compared with the FP64 ones relative to their largest component; checkpoint
spacing must not change the result (the recomputed iterates are the same computation).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1609_05722_gb300 import build as B_  # noqa: E402
from paper_1609_05722_gb300 import foe as F  # noqa: E402
from paper_1609_05722_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
F32 = np.float32


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B_.build()
    torch.cuda.set_device(0)
    k, a = synth.filter_bank()
    return k.astype(F32), a.astype(F32)


def batch(Bn, H, W, peak, seed):
    ld = (W + 3) // 4 * 4
    clean = np.stack([synth.clean_image(H, W, seed + s) * peak for s in range(Bn)])
    noisy = np.stack([synth.poisson_observation(clean[s] / peak, peak, seed + 100 + s) for s in range(Bn)])
    cd = torch.zeros((Bn, H, ld), dtype=torch.float32, device="cuda")
    nd = torch.zeros((Bn, H, ld), dtype=torch.float32, device="cuda")
    cd[:, :, :W] = torch.from_numpy(clean.astype(F32)).cuda()
    nd[:, :, :W] = torch.from_numpy(noisy.astype(F32)).cuda()
    return clean, noisy, cd, nd, ld


def gpu_grad(ctx, cd, nd, Bn, H, W, ld, T, tau, bc, ckpt):
    dk = torch.zeros((48, 49), dtype=torch.float32, device="cuda")
    da = torch.zeros((48,), dtype=torch.float32, device="cuda")
    opts = F.SolveOpts(model=F.FOE_MODEL_ANS_L2, prec=F.FOE_PREC_FP32, iters=T, tau=tau, bc=bc, lam=1.0,
                       gamma=float(F32(0.8)))
    L = F.foe_train_step(ctx, cd, nd, Bn, H, W, ld, opts, dk, da, ckpt)
    torch.cuda.synchronize()
    return L, dk.cpu().numpy().astype(np.float64).reshape(48, 7, 7), da.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("shape,bc", [((24, 24), F.FOE_BC_SYMMETRIC), ((37, 45), F.FOE_BC_ZERO),
                                      ((40, 33), F.FOE_BC_SYMMETRIC)])
def test_gradient_matches_oracle(setup, shape, bc):
    k, a = setup
    H, W = shape
    Bn, T = 3, 8
    clean, noisy, cd, nd, ld = batch(Bn, H, W, 4.0, 500 + H)
    ctx = F.foe_create(k, a)
    try:
        tau = float(F32(0.01))
        L, dk, da = gpu_grad(ctx, cd, nd, Bn, H, W, ld, T, tau, bc, 3)
    finally:
        F.foe_destroy(ctx)
    pr = O.Problem(k.astype(np.float64), a.astype(np.float64), H, W, bc=bc, model=O.MODEL_ANS_L2, lam=1.0, tau=tau,
                   gamma=float(F32(0.8)))
    Lr, dkr, dar = pr.train_grad(clean, noisy, T)
    assert L == pytest.approx(Lr, rel=1e-5)
    assert np.abs(dk - dkr).max() <= 2e-4 * np.abs(dkr).max()
    assert np.abs(da - dar).max() <= 2e-4 * np.abs(dar).max()


def test_checkpoint_spacing_does_not_change_the_gradient(setup):
    k, a = setup
    H, W, Bn, T = 30, 30, 2, 7
    _, _, cd, nd, ld = batch(Bn, H, W, 4.0, 700)
    ctx = F.foe_create(k, a)
    try:
        res = [gpu_grad(ctx, cd, nd, Bn, H, W, ld, T, 0.01, F.FOE_BC_SYMMETRIC, c) for c in (1, 3, 7)]
    finally:
        F.foe_destroy(ctx)
    for L, dk, da in res[1:]:
        assert L == res[0][0]
        assert np.array_equal(dk, res[0][1]) and np.array_equal(da, res[0][2])


def test_config_size_subbatch_against_oracle(setup):
    # 180x180 images, peak 4, 50 checkpointed iterations (the training configuration), 2-image sub-batch
    k, a = setup
    H = W = 180
    Bn, T = 2, 50
    clean, noisy, cd, nd, ld = batch(Bn, H, W, 4.0, 900)
    ctx = F.foe_create(k, a)
    try:
        tau, _ = F.foe_step_size(ctx, F.FOE_BC_SYMMETRIC, float(F32(0.8)))
        L, dk, da = gpu_grad(ctx, cd, nd, Bn, H, W, ld, T, tau, F.FOE_BC_SYMMETRIC, 0)
    finally:
        F.foe_destroy(ctx)
    pr = O.Problem(k.astype(np.float64), a.astype(np.float64), H, W, model=O.MODEL_ANS_L2, lam=1.0, tau=tau,
                   gamma=float(F32(0.8)))
    Lr, dkr, dar = pr.train_grad(clean, noisy, T)
    assert L == pytest.approx(Lr, rel=1e-5)
    assert np.abs(dk - dkr).max() <= 1e-3 * np.abs(dkr).max()
    assert np.abs(da - dar).max() <= 1e-3 * np.abs(dar).max()


def test_autograd_function(setup):
    from paper_1609_05722_gb300.train import FoEUnrolledLoss
    k, a = setup
    H = W = 28
    _, _, cd, nd, ld = batch(2, H, W, 4.0, 800)
    filt = torch.tensor(k, requires_grad=True)
    la = torch.tensor(np.log(a), requires_grad=True)
    loss = FoEUnrolledLoss.apply(filt, la, cd, nd, 6, 1.0, float(F32(0.8)), 0.01, 0, W)
    (2.0 * loss).backward()
    ctx = F.foe_create(k, a)
    try:
        L, dk, da = gpu_grad(ctx, cd, nd, 2, H, W, ld, 6, 0.01, F.FOE_BC_SYMMETRIC, 0)
    finally:
        F.foe_destroy(ctx)
    assert float(loss.detach()) == pytest.approx(L, rel=1e-12)
    np.testing.assert_allclose(filt.grad.numpy(), 2.0 * dk, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(la.grad.numpy(), 2.0 * da, rtol=1e-6, atol=1e-6)
