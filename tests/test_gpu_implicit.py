"""The paper's training gradient by implicit differentiation (Sec. 2.5, Eq. implicitdifferentiation and Eq.
overallderivative), foe_train_grad_implicit, against the FP64 oracle (itself pinned by central differences of the
converged loss, a dense solve and the unrolled gradient at large T in the oracle tests).

The device solves H_E q = dL/dw by conjugate gradients on FP32 vectors (FP64 dot products): its true residual
stalls near cond(H_E) times the FP32 unit roundoff; the gradients, sums of many products with q, land far closer
(a few 1e-6 measured), and are compared with those of the oracle's tightly solved q relative to their largest
component at 1e-4.
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
GAMMA = float(F32(0.8))


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B_.build()
    torch.cuda.set_device(0)
    k, a = synth.filter_bank()
    k, a = k.astype(F32), a.astype(F32)
    ctx = F.foe_create(k, a)
    yield k, a, ctx
    F.foe_destroy(ctx)


def batch(Bn, H, W, peak, seed):
    ld = (W + 3) // 4 * 4
    clean = np.stack([synth.clean_image(H, W, seed + s) * peak for s in range(Bn)])
    noisy = np.stack([synth.poisson_observation(clean[s] / peak, peak, seed + 100 + s) for s in range(Bn)])
    cd = torch.zeros((Bn, H, ld), dtype=torch.float32, device="cuda")
    nd = torch.zeros((Bn, H, ld), dtype=torch.float32, device="cuda")
    cd[:, :, :W] = torch.from_numpy(clean.astype(F32)).cuda()
    nd[:, :, :W] = torch.from_numpy(noisy.astype(F32)).cuda()
    return clean, noisy, cd, nd, ld


def opts(T, tau, bc, lam=1.0):
    return F.SolveOpts(model=F.FOE_MODEL_ANS_L2, prec=F.FOE_PREC_FP32, iters=T, tau=tau, bc=bc, lam=lam, gamma=GAMMA)


def implicit(ctx, cd, nd, Bn, H, W, ld, T, tau, bc, max_cg=500, tol=1e-5, lam=1.0):
    dk = torch.zeros((48, 49), dtype=torch.float32, device="cuda")
    da = torch.zeros((48,), dtype=torch.float32, device="cuda")
    L, rep = F.foe_train_grad_implicit(ctx, cd, nd, Bn, H, W, ld, opts(T, tau, bc, lam), dk, da, max_cg, tol)
    torch.cuda.synchronize()
    return L, dk.cpu().numpy().astype(np.float64).reshape(48, 7, 7), da.cpu().numpy().astype(np.float64), rep


# lambda = 5 under zero padding: with lambda = 1 the zero-extended prior pulls this image below the clamp of the
# output map everywhere within 150 steps, where dL/dw (and every gradient) vanishes
@pytest.mark.parametrize("shape,bc,lam", [((24, 24), F.FOE_BC_SYMMETRIC, 1.0), ((37, 45), F.FOE_BC_ZERO, 5.0),
                                          ((40, 33), F.FOE_BC_SYMMETRIC, 1.0)])
def test_implicit_gradient_matches_oracle(setup, shape, bc, lam):
    k, a, ctx = setup
    H, W = shape
    Bn, T = 2, 150
    clean, noisy, cd, nd, ld = batch(Bn, H, W, 4.0, 800 + H)
    tau, _ = F.foe_step_size(ctx, bc, GAMMA)
    L, dk, da, rep = implicit(ctx, cd, nd, Bn, H, W, ld, T, tau, bc, lam=lam)
    pr = O.Problem(k.astype(np.float64), a.astype(np.float64), H, W, bc=bc, model=O.MODEL_ANS_L2, lam=lam, tau=tau,
                   gamma=GAMMA)
    Lr, dkr, dar, itr, relr = pr.train_grad_implicit(clean, noisy, T, 2000, 1e-12)
    assert itr > 0
    ek = np.abs(dk - dkr).max() / np.abs(dkr).max()
    ea = np.abs(da - dar).max() / np.abs(dar).max()
    print(f"implicit {shape} bc={bc}: CG {rep['cg_iters']} it (oracle {itr}), relres {rep['cg_relres']:.1e}; "
          f"dk err {ek:.1e}, dlogalpha err {ea:.1e}")
    assert rep["breakdowns"] == 0 and rep["cg_relres"] <= 1e-5
    assert L == pytest.approx(Lr, rel=1e-5)
    assert ek <= 1e-4 and ea <= 1e-4


def test_implicit_equals_unrolled_gradient_when_the_solve_has_converged(setup):
    # the two routes to dL/dtheta agree once u^T is at the minimiser (oracle pin at T = 3000 on 8x9; here on the
    # device, 24x28 images, T = 1200)
    k, a, ctx = setup
    H, W, Bn, T = 24, 28, 2, 1200
    _, _, cd, nd, ld = batch(Bn, H, W, 4.0, 900)
    tau, _ = F.foe_step_size(ctx, F.FOE_BC_SYMMETRIC, GAMMA)
    L, dk, da, rep = implicit(ctx, cd, nd, Bn, H, W, ld, T, tau, F.FOE_BC_SYMMETRIC)
    dku = torch.zeros((48, 49), dtype=torch.float32, device="cuda")
    dau = torch.zeros((48,), dtype=torch.float32, device="cuda")
    Lu = F.foe_train_step(ctx, cd, nd, Bn, H, W, ld, opts(T, tau, F.FOE_BC_SYMMETRIC), dku, dau, 0)
    torch.cuda.synchronize()
    dku = dku.cpu().numpy().astype(np.float64).reshape(48, 7, 7)
    dau = dau.cpu().numpy().astype(np.float64)
    ek = np.abs(dk - dku).max() / np.abs(dku).max()
    ea = np.abs(da - dau).max() / np.abs(dau).max()
    print(f"implicit vs unrolled at T={T}: dk {ek:.1e}, dlogalpha {ea:.1e}; CG {rep['cg_iters']} it")
    assert L == pytest.approx(Lu, rel=1e-6)
    assert ek <= 2e-4 and ea <= 2e-4


def test_implicit_rejects_unsupported_options(setup):
    k, a, ctx = setup
    cd = torch.zeros((1, 16, 16), device="cuda")
    dk = torch.zeros((48, 49), device="cuda")
    da = torch.zeros((48,), device="cuda")
    bad = F.SolveOpts(model=F.FOE_MODEL_ANS_IDIV, prec=F.FOE_PREC_FP32, iters=5)
    with pytest.raises(F.FoeError) as e:
        F.foe_train_grad_implicit(ctx, cd, cd, 1, 16, 16, 16, bad, dk, da)
    assert e.value.status == F.FOE_EUNSUPPORTED
    with pytest.raises(F.FoeError) as e:
        F.foe_train_grad_implicit(ctx, cd, cd, 1, 16, 16, 16, opts(5, 0.0, F.FOE_BC_SYMMETRIC), dk, da, max_cg=0)
    assert e.value.status == F.FOE_EINVAL


def test_lbfgs_training_with_the_implicit_gradient_decreases_the_loss(setup):
    # Algorithm 1 on the device: a few L-BFGS iterations over all 48 filters and log-weights on a small batch
    from paper_1609_05722_gb300.train import FoEImplicitLoss, lbfgs_train
    k, a, _ = setup
    H, W, Bn = 32, 32, 2
    _, _, cd, nd, ld = batch(Bn, H, W, 4.0, 950)

    def loss_fn(kt, lat):
        return FoEImplicitLoss.apply(kt, lat, cd, nd, 300, 1.0, GAMMA, 0.0, 300, 1e-5, W)

    kt, lat, losses, reason = lbfgs_train(loss_fn, torch.from_numpy(k.astype(np.float64)).view(48, 7, 7),
                                          torch.from_numpy(np.log(a.astype(np.float64))), max_iter=3, tol=0.0)
    print(f"L-BFGS (implicit gradient) losses {[round(x, 4) for x in losses]} ({reason})")
    assert losses[1] < losses[0] and min(losses) < 0.999 * losses[0]


def test_lbfgs_on_the_device_follows_the_oracle_driven_trajectory(setup):
    # Algorithm 1 driven by the device's loss and implicit gradient against the same driver given the FP64 oracle's
    # (6 filters, two 8x9 images at peak 4, 400 inner iterations, the step of each evaluation's filters): the losses
    # of the iterations agree to 1e-4 relative and the parameters end within 1 % of the distance they moved.
    from paper_1609_05722_gb300.train import FoEImplicitLoss, lbfgs_train
    k, a, _ = setup
    NF, H, W, Bn, T = 6, 8, 9, 2, 400
    clean, noisy, cd, nd, ld = batch(Bn, H, W, 4.0, 70)

    class OracleLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, kt, lat):
            kk = kt.detach().numpy()
            aa = np.exp(lat.detach().numpy())
            tau = 0.99 * 2 * (1 - GAMMA) / (O.lipschitz(kk, aa) + 2e-3)
            pr = O.Problem(kk, aa, H, W, model=O.MODEL_ANS_L2, lam=1.0, tau=tau, gamma=GAMMA, nthreads=1)
            L, dk, da, _, _ = pr.train_grad_implicit(clean, noisy, T, 500, 1e-10)
            ctx.save_for_backward(torch.from_numpy(dk), torch.from_numpy(da))
            return torch.tensor(L, dtype=torch.float64)

        @staticmethod
        def backward(ctx, g):
            dk, da = ctx.saved_tensors
            return g * dk, g * da

    def device_loss(kt, lat):
        return FoEImplicitLoss.apply(kt, lat, cd, nd, T, 1.0, GAMMA, 0.0, 500, 1e-5, W)

    k0 = torch.from_numpy(k[:NF].astype(np.float64)).view(NF, 7, 7)
    la0 = torch.from_numpy(np.log(a[:NF].astype(np.float64)))
    kd, lad, Ld, rd = lbfgs_train(device_loss, k0.clone(), la0.clone(), max_iter=3, tol=0.0)
    ko, lao, Lo, ro = lbfgs_train(OracleLoss.apply, k0.clone(), la0.clone(), max_iter=3, tol=0.0)
    print(f"L-BFGS device {[round(x, 6) for x in Ld]} ({rd}), oracle {[round(x, 6) for x in Lo]} ({ro})")
    assert rd == ro == "max_iter" and len(Ld) == len(Lo) == 4
    np.testing.assert_allclose(Ld, Lo, rtol=1e-4)
    assert Lo[-1] < 0.99 * Lo[0]
    assert torch.linalg.vector_norm(kd - ko) <= 1e-2 * torch.linalg.vector_norm(ko - k0)
    assert torch.linalg.vector_norm(lad - lao) <= 1e-2 * torch.linalg.vector_norm(lao - la0)


@pytest.mark.parametrize("shape,bc", [((40, 33), F.FOE_BC_SYMMETRIC), ((64, 60), F.FOE_BC_ZERO)])
def test_implicit_gradient_with_tensor_core_hessian_products(setup, shape, bc):
    # opts.prec = TF32: the CG's Hessian-vector products on the tensor cores (TF32 operands: the direction's
    # responses and the curvature-weighted products are rounded to 10-bit mantissas, about 5e-4 each), the rest
    # FP32.  The gradients follow the oracle's to 1e-3 of their largest component (measured 2e-4), the loss exactly as
    # the FP32 path
    # (the same lower-level solve), and the CG converges on the TF32 operator.
    k, a, ctx = setup
    H, W = shape
    Bn, T = 2, 150
    clean, noisy, cd, nd, ld = batch(Bn, H, W, 4.0, 850 + H)
    tau, _ = F.foe_step_size(ctx, bc, GAMMA)
    L32, dk32, da32, rep32 = implicit(ctx, cd, nd, Bn, H, W, ld, T, tau, bc)
    dk = torch.zeros((48, 49), dtype=torch.float32, device="cuda")
    da = torch.zeros((48,), dtype=torch.float32, device="cuda")
    o = F.SolveOpts(model=F.FOE_MODEL_ANS_L2, prec=F.FOE_PREC_TF32, iters=T, tau=tau, bc=bc, lam=1.0, gamma=GAMMA)
    L, rep = F.foe_train_grad_implicit(ctx, cd, nd, Bn, H, W, ld, o, dk, da, 500, 1e-5)
    torch.cuda.synchronize()
    dk = dk.cpu().numpy().astype(np.float64).reshape(48, 7, 7)
    da = da.cpu().numpy().astype(np.float64)
    pr = O.Problem(k.astype(np.float64), a.astype(np.float64), H, W, bc=bc, model=O.MODEL_ANS_L2, lam=1.0, tau=tau,
                   gamma=GAMMA)
    Lr, dkr, dar, _, _ = pr.train_grad_implicit(clean, noisy, T, 2000, 1e-12)
    ek = np.abs(dk - dkr).max() / np.abs(dkr).max()
    ea = np.abs(da - dar).max() / np.abs(dar).max()
    print(f"implicit TF32 {shape} bc={bc}: CG {rep['cg_iters']} it (FP32 {rep32['cg_iters']}), relres "
          f"{rep['cg_relres']:.1e}; dk err {ek:.1e}, dlogalpha err {ea:.1e}")
    assert L == L32 and L == pytest.approx(Lr, rel=1e-5)
    assert rep["breakdowns"] == 0 and rep["cg_relres"] <= 1e-5
    assert ek <= 1e-3 and ea <= 1e-3
