"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

The oracle is given exactly the parameters the GPU sees (filters, weights, tau, gamma and lambda
rounded to FP32 first).  Tolerances:
  * one plain-FP32 step / gradient: the FP32 gradient's rounding (relative ~1e-6 of |g|) times tau;
  * whole plain-FP32 solves: max-abs <= 1e-4 on the [0, 255]-scaled output (255 / peak scaling);
  * BF16 tensor-core solves: PSNR within 0.02 dB of the oracle's PSNR against the clean image.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1609_05722_gb300 import build as B  # noqa: E402
from paper_1609_05722_gb300 import foe as F  # noqa: E402
from paper_1609_05722_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

F32 = np.float32
GAMMA = float(F32(0.8))
LAM = 1.0


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


@pytest.fixture(scope="module")
def bank32(bank):
    k, a = bank
    return k.astype(F32), a.astype(F32)


@pytest.fixture(scope="module")
def ctx(dev, bank32):
    c = F.foe_create(*bank32)
    yield c
    F.foe_destroy(c)


def ld_of(W):
    return (W + 3) // 4 * 4


def to_dev(a, dev, ld=None):
    a = np.asarray(a, dtype=F32)
    H, W = a.shape
    ld = ld or ld_of(W)
    t = torch.zeros((H, ld), dtype=torch.float32, device=dev)
    t[:, :W] = torch.from_numpy(np.ascontiguousarray(a))
    return t


def from_dev(t, W):
    return t[:, :W].double().cpu().numpy()


def problem(bank32, H, W, model, bc, tau, nthreads=None):
    k, a = bank32
    return O.Problem(k.astype(np.float64), a.astype(np.float64), H, W, bc=bc, model=model, lam=LAM, tau=tau,
                     gamma=GAMMA, nthreads=nthreads)


def data_for(model, H, W, peak, seed):
    y = synth.poisson_observation(synth.clean_image(H, W, seed), peak, seed + 1)
    d = y if model == O.MODEL_DIRECT else O.anscombe(y)
    return y, d


# ----------------------------------------------------------------------------- elementwise

def test_anscombe_and_inverse(dev):
    rng = np.random.default_rng(0)
    y = rng.integers(0, 200, 5000).astype(F32)
    yd = torch.tensor(y, device=dev)
    vd = torch.empty_like(yd)
    F.foe_anscombe(yd, vd, y.size)
    ref = O.anscombe(y.astype(np.float64)).astype(F32)
    np.testing.assert_array_equal(vd.cpu().numpy(), ref)  # FP64 on both sides, rounded once
    z = rng.uniform(0.3, 30.0, 5000).astype(F32)
    zd = torch.tensor(z, device=dev)
    xd = torch.empty_like(zd)
    F.foe_inverse(zd, xd, z.size)
    ref = O.inverse(z.astype(np.float64))
    np.testing.assert_allclose(xd.cpu().numpy(), ref, rtol=2e-7, atol=1e-7)


# ----------------------------------------------------------------------------- one step, FP32

SHAPES = [(64, 64), (13, 17), (37, 70), (96, 33), (7, 7)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", [F.FOE_BC_SYMMETRIC, F.FOE_BC_ZERO])
@pytest.mark.parametrize("model", [F.FOE_MODEL_DIRECT, F.FOE_MODEL_ANS_L2, F.FOE_MODEL_ANS_IDIV])
def test_single_step_fp32(dev, ctx, bank32, shape, bc, model):
    H, W = shape
    tau, _ = F.foe_step_size(ctx, bc, GAMMA)
    y, d = data_for(model, H, W, 6.0, 100 + H)
    rng = np.random.default_rng(H * W)
    u = (d + rng.uniform(-0.3, 0.3, d.shape)).clip(0.05).astype(F32).astype(np.float64)
    delta = rng.uniform(-0.05, 0.05, d.shape).astype(F32).astype(np.float64)
    d32 = d.astype(F32).astype(np.float64)
    pr = problem(bank32, H, W, model, bc, tau)
    ref = pr.step(d32, u, u - delta)
    uh, dl, dd = to_dev(u, dev), to_dev(delta, dev), to_dev(d32, dev)
    ul = torch.zeros_like(uh)
    un = torch.zeros_like(uh)
    F.foe_ipiano_step(ctx, uh, ul, dl, dd, un, H, W, uh.shape[1], model, LAM, tau, GAMMA, bc, F.FOE_PREC_FP32)
    torch.cuda.synchronize()
    got = from_dev(un, W) + from_dev(ul, W)
    assert np.abs(got - ref).max() <= 2e-6
    np.testing.assert_allclose(from_dev(dl, W), ref - u, atol=2e-6)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", [F.FOE_BC_SYMMETRIC, F.FOE_BC_ZERO])
@pytest.mark.parametrize("model", [F.FOE_MODEL_DIRECT, F.FOE_MODEL_ANS_L2, F.FOE_MODEL_ANS_IDIV])
def test_energy_and_gradient_fp32(dev, ctx, bank32, shape, bc, model):
    H, W = shape
    y, d = data_for(model, H, W, 5.0, 200 + W)
    rng = np.random.default_rng(7 * H + W)
    u = (d + rng.uniform(-0.5, 0.5, d.shape)).clip(0.1).astype(F32).astype(np.float64)
    d32 = d.astype(F32).astype(np.float64)
    pr = problem(bank32, H, W, model, bc, 1e-3)
    e_ref, g_ref = pr.energy_grad(u, d32)
    ud, dd = to_dev(u, dev), to_dev(d32, dev)
    gd = torch.zeros_like(ud)
    e = F.foe_energy_grad(ctx, ud, dd, H, W, ud.shape[1], model, LAM, bc, F.FOE_PREC_FP32, grad=gd)
    g = from_dev(gd, W)
    assert np.abs(g - g_ref).max() <= 2e-5 * max(1.0, np.abs(g_ref).max())
    assert e == pytest.approx(e_ref, rel=2e-6)


# ----------------------------------------------------------------------------- whole solves, FP32

def run_denoise(dev, ctx, y, peak, opts):
    H, W = y.shape
    yd = to_dev(y, dev)
    xd = torch.zeros_like(yd)
    rep = F.foe_denoise(ctx, yd, xd, H, W, yd.shape[1], peak, opts, report=True)
    return from_dev(xd, W), rep


@pytest.mark.parametrize("model", [F.FOE_MODEL_ANS_L2, F.FOE_MODEL_DIRECT, F.FOE_MODEL_ANS_IDIV, F.FOE_MODEL_AUTO])
def test_denoise_fp32_64x64_100_iterations(dev, ctx, bank32, model):
    # 64x64, peak 4, 100 iterations: plain-FP32 max-abs <= 1e-4 on the [0, 255] scale.
    H = W = 64
    peak = 4.0
    clean = synth.clean_image(H, W, 1000)
    y = synth.poisson_observation(clean, peak, 5000)
    tau, _ = F.foe_step_size(ctx, F.FOE_BC_SYMMETRIC, GAMMA)
    opts = F.SolveOpts(model=model, iters=100, prec=F.FOE_PREC_FP32, tau=tau)
    x, rep = run_denoise(dev, ctx, y, peak, opts)
    used = rep["model_used"]
    ref, used_ref = problem(bank32, H, W, model, F.FOE_BC_SYMMETRIC, tau).denoise(y, peak, 100)
    assert used == used_ref
    err = np.abs(x - ref).max() * 255.0 / peak
    assert err <= 1e-4, err


@pytest.mark.parametrize("shape,bc,peak", [((37, 70), F.FOE_BC_ZERO, 2.0), ((50, 9), F.FOE_BC_SYMMETRIC, 30.0),
                                           ((100, 131), F.FOE_BC_SYMMETRIC, 1.0)])
def test_denoise_fp32_ragged(dev, ctx, bank32, shape, bc, peak):
    H, W = shape
    y = synth.poisson_observation(synth.clean_image(H, W, 77), peak, 78)
    tau, _ = F.foe_step_size(ctx, bc, GAMMA)
    opts = F.SolveOpts(model=F.FOE_MODEL_AUTO, iters=60, prec=F.FOE_PREC_FP32, tau=tau, bc=bc)
    x, rep = run_denoise(dev, ctx, y, peak, opts)
    ref, _ = problem(bank32, H, W, F.FOE_MODEL_AUTO, bc, tau).denoise(y, peak, 60)
    assert np.abs(x - ref).max() * 255.0 / peak <= 1e-4


def test_denoise_fp32_zero_iterations_and_zero_replacement(dev, ctx, bank32):
    H, W = 20, 24
    y = synth.poisson_observation(synth.clean_image(H, W, 5), 1.0, 6)
    tau, _ = F.foe_step_size(ctx, F.FOE_BC_SYMMETRIC, GAMMA)
    for model in (F.FOE_MODEL_DIRECT, F.FOE_MODEL_ANS_L2):
        opts = F.SolveOpts(model=model, iters=0, prec=F.FOE_PREC_FP32, tau=tau, zero_c=0.1)
        x, _ = run_denoise(dev, ctx, y, 1.0, opts)
        ref, _ = problem(bank32, H, W, model, F.FOE_BC_SYMMETRIC, tau).denoise(y, 1.0, 0, zero_c=float(F32(0.1)))
        np.testing.assert_allclose(x, ref, rtol=1e-7, atol=1e-7)


@pytest.mark.parametrize("model,peak", [(F.FOE_MODEL_ANS_L2, 4.0), (F.FOE_MODEL_DIRECT, 30.0)])
def test_denoise_fp32_512_full(dev, ctx, bank32, model, peak):
    # The benchmark size: 512x512, 300 iterations, every output pixel against the oracle.
    H = W = 512
    clean = synth.clean_image(H, W, 1000) * peak
    y = synth.poisson_observation(clean / peak, peak, 5000)
    tau, _ = F.foe_step_size(ctx, F.FOE_BC_SYMMETRIC, GAMMA)
    opts = F.SolveOpts(model=model, iters=300, prec=F.FOE_PREC_FP32, tau=tau)
    x, _ = run_denoise(dev, ctx, y, peak, opts)
    ref, _ = problem(bank32, H, W, model, F.FOE_BC_SYMMETRIC, tau).denoise(y, peak, 300)
    assert np.abs(x - ref).max() * 255.0 / peak <= 1e-4
    assert abs(O.psnr(x, clean, peak) - O.psnr(ref, clean, peak)) <= 1e-3


# ----------------------------------------------------------------------------- batch == single

def test_batch_equals_single_images(dev, ctx):
    specs = [(64, 64, 4.0, 30), (37, 70, 12.0, 45), (128, 96, 2.0, 10), (9, 200, 30.0, 0)]
    ys, xs, descs, singles = [], [], [], []
    for j, (H, W, peak, it) in enumerate(specs):
        y = synth.poisson_observation(synth.clean_image(H, W, 300 + j), peak, 400 + j)
        yd = to_dev(y, dev)
        xd = torch.zeros_like(yd)
        ys.append(yd)
        xs.append(xd)
        descs.append({"y": yd, "x": xd, "H": H, "W": W, "ld": yd.shape[1], "peak": peak, "iters": it})
    opts = F.SolveOpts(model=F.FOE_MODEL_AUTO, prec=F.FOE_PREC_FP32)
    F.foe_denoise_batch(ctx, descs, opts)
    for j, (H, W, peak, it) in enumerate(specs):
        xd = torch.zeros_like(ys[j])
        o = F.SolveOpts(model=F.FOE_MODEL_AUTO, prec=F.FOE_PREC_FP32, iters=it)
        F.foe_denoise(ctx, ys[j], xd, H, W, ys[j].shape[1], peak, o)
        singles.append(xd)
    torch.cuda.synchronize()
    for j in range(len(specs)):
        assert torch.equal(xs[j], singles[j]), j


def test_repeat_runs_are_bitwise_identical(dev, ctx):
    H, W = 70, 90
    y = synth.poisson_observation(synth.clean_image(H, W, 9), 3.0, 10)
    opts = F.SolveOpts(model=F.FOE_MODEL_AUTO, iters=25, prec=F.FOE_PREC_FP32)
    a, _ = run_denoise(dev, ctx, y, 3.0, opts)
    b, _ = run_denoise(dev, ctx, y, 3.0, opts)
    assert np.array_equal(a, b)
