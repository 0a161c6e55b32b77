"""The binning variant FoEPNRbin (Sec. 4: 3x3 ones-kernel bins, solve at nine times the peak, bilinear upscaling)
through foe_denoise_binned, against the FP64 oracle.

The bin sums are exact (integer counts) up to the 9 / n scaling of border bins and the upscaling is one FP32
weighted sum, so the two together agree with the oracle to a few 1e-7 relative; the solve on the bin image is held
to the FP32 path's bar (max-abs 1e-4 on the 255 scale) and, on the tensor-core paths, to the metric's bar,
|PSNR(gpu) - PSNR(oracle)| <= 0.02 dB against the clean image.
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


@pytest.fixture(scope="module")
def bank32(bank):
    k, a = bank
    return k.astype(F32), a.astype(F32)


@pytest.fixture(scope="module")
def ctx(bank32):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    torch.cuda.set_device(0)
    c = F.foe_create(*bank32)
    yield c
    F.foe_destroy(c)


def _run(ctx, y, peak, opts, report=False):
    H, W = y.shape
    ld = (W + 3) // 4 * 4
    yd = torch.zeros((H, ld), dtype=torch.float32, device="cuda")
    yd[:, :W] = torch.from_numpy(y.astype(F32))
    xd = torch.full_like(yd, -1.0)
    rep = F.foe_denoise_binned(ctx, yd, xd, H, W, ld, peak, opts, report=report)
    torch.cuda.synchronize()
    return xd[:, :W].double().cpu().numpy(), rep


@pytest.mark.parametrize("shape", [(19, 19), (61, 70), (100, 101), (64, 66)])
def test_bins_and_upscaling_without_iterations(ctx, shape):
    # direct data term, no iterations: the estimate of the bin image is the bin image itself, so the result is the
    # oracle's upscale3(bin3(y)) (every border case of both maps: 19 = 3 * 6 + 1, 70 = 3 * 23 + 1, 101 = 3 * 33 + 2)
    H, W = shape
    y = np.random.default_rng(H * 1000 + W).poisson(2.5, (H, W)).astype(np.float64)
    x, _ = _run(ctx, y, 2.5, F.SolveOpts(model=F.FOE_MODEL_DIRECT, iters=0, prec=F.FOE_PREC_FP32))
    ref = O.upscale3(O.bin3(y), H, W)
    err = np.abs(x - ref).max() / np.abs(ref).max()
    print(f"bin/upscale {shape}: max rel {err:.2e}")
    assert err <= 1e-6


@pytest.mark.parametrize("model,peak,shape", [(F.FOE_MODEL_ANS_L2, 1.0, (64, 70)), (F.FOE_MODEL_DIRECT, 2.0, (61, 53)),
                                              (F.FOE_MODEL_ANS_IDIV, 0.4, (57, 64)), (F.FOE_MODEL_AUTO, 0.3, (48, 50)),
                                              (F.FOE_MODEL_AUTO, 0.7, (40, 44))])
def test_binned_fp32_matches_oracle(ctx, bank32, model, peak, shape):
    H, W = shape
    iters = 60
    clean = synth.clean_image(H, W, 40 + H) * peak
    y = synth.poisson_observation(clean / peak, peak, 41 + W)
    tau, _ = F.foe_step_size(ctx, F.FOE_BC_SYMMETRIC, GAMMA)
    x, rep = _run(ctx, y, peak, F.SolveOpts(model=model, iters=iters, prec=F.FOE_PREC_FP32, tau=tau, gamma=GAMMA),
                  report=True)
    k, a = bank32
    pr = O.Problem(k.astype(np.float64), a.astype(np.float64), H, W, model=model, lam=1.0, tau=tau, gamma=GAMMA)
    ref, used = pr.denoise_binned(y, peak, iters)
    assert rep["model_used"] == used
    err = np.abs(x - ref).max() * 255.0 / peak
    print(f"binned fp32 model={model} peak={peak} {shape} (binned model {used}): max-abs {err:.2e} on the 255 scale")
    assert err <= 1e-4


@pytest.mark.parametrize("prec", [F.FOE_PREC_BF16, F.FOE_PREC_TF32])
def test_binned_512_psnr_vs_oracle(ctx, bank32, prec):
    # the regime the paper bins in (peak < 1): 512 x 512 at peak 0.5, so the bin image (171 x 171, 512 = 3 * 170 + 2)
    # has peak 4.5 and the I-divergence data term; 300 iterations
    H = W = 512
    peak = 0.5
    clean = synth.clean_image(H, W, 1200) * peak
    y = synth.poisson_observation(clean / peak, peak, 6200)
    tau, _ = F.foe_step_size(ctx, F.FOE_BC_SYMMETRIC, GAMMA)
    opts = F.SolveOpts(model=F.FOE_MODEL_AUTO, iters=300, prec=prec, tau=tau, gamma=GAMMA)
    x, rep = _run(ctx, y, peak, opts, report=True)
    k, a = bank32
    pr = O.Problem(k.astype(np.float64), a.astype(np.float64), H, W, model=O.MODEL_AUTO, lam=1.0, tau=tau,
                   gamma=GAMMA)
    ref, used = pr.denoise_binned(y, peak, 300)
    assert used == O.MODEL_ANS_IDIV and rep["model_used"] == used
    p_gpu, p_ref = O.psnr(x, clean, peak), O.psnr(ref, clean, peak)
    print(f"binned 512 prec={prec}: PSNR {p_gpu:.3f} dB vs oracle {p_ref:.3f} dB (dPSNR {abs(p_gpu - p_ref):.4f})")
    assert abs(p_gpu - p_ref) <= 0.02


def test_binned_rejects_images_whose_bin_image_is_below_7x7(ctx):
    y = torch.ones((18, 20), device="cuda")
    x = torch.zeros_like(y)
    with pytest.raises(F.FoeError) as e:
        F.foe_denoise_binned(ctx, y, x, 18, 20, 20, 1.0, F.SolveOpts(prec=F.FOE_PREC_FP32))
    assert e.value.status == F.FOE_EINVAL
