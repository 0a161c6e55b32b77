"""Tensor-core (tcgen05, BF16 or TF32 operands, FP32 accumulation) paths vs the FP64 oracle.

Tolerances follow from the arithmetic: u, the filters and psi are rounded to BF16 (relative 2^-9) or
TF32 (2^-11), so one gradient differs from the exact one by at most a few 1e-3 of its scale (BF16);
a whole solve is held to the metric's bar, |PSNR(tc) - PSNR(oracle)| <= 0.02 dB against the clean
image.
"""
import json
import os

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
BF16 = F.FOE_PREC_BF16
TF32 = F.FOE_PREC_TF32
TC_PRECS = [BF16, TF32]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_512.json")


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


def to_dev(a, dev):
    a = np.asarray(a, dtype=F32)
    H, W = a.shape
    ld = (W + 3) // 4 * 4
    t = torch.zeros((H, ld), dtype=torch.float32, device=dev)
    t[:, :W] = torch.from_numpy(np.ascontiguousarray(a))
    return t


def from_dev(t, W):
    return t[:, :W].double().cpu().numpy()


def problem(bank32, H, W, model, bc, tau):
    k, a = bank32
    return O.Problem(k.astype(np.float64), a.astype(np.float64), H, W, bc=bc, model=model, lam=LAM, tau=tau,
                     gamma=GAMMA)


# Images below 90000 pixels or 59 rows (and every TF32 image) take 26 x 26 tiles: widths 54 and 79 leave a last tile
# of 2 and 1 columns after full 26-column tiles, where the reflection of a pixel within 3 columns of the right border
# falls outside a 32-column response region that does not reach it; width 28 puts the flush last tile at column 2,
# so the columns within 3 of the left border must stay with the first tile.  Larger BF16 images (at least 67 rows)
# take the pixel-pair tiles of 58 columns x 66 rows (PAIR_SHAPES, long strips so that the small side sets the case):
# 59 / 60 columns and 67 / 68 rows put the flush last tile at 1 / 2 (the same split rule in both directions), 117,
# 122, 135 and 456 leave ragged flush tiles, 30 and 33 columns are narrower than one tile.
PAIR_SHAPES = [(3440, 59), (67, 3000), (3335, 60), (68, 2950), (1720, 117), (122, 1650), (6700, 30), (6100, 33),
               (456, 456), (135, 1490)]
SHAPES = [(64, 64), (13, 17), (37, 70), (96, 33), (7, 7), (130, 200), (53, 54), (28, 79), (240, 70), (233, 30),
          (40, 28), (59, 60), (60, 59), (61, 122), (120, 117), (116, 59)] + PAIR_SHAPES


@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", [F.FOE_BC_SYMMETRIC, F.FOE_BC_ZERO])
@pytest.mark.parametrize("model", [F.FOE_MODEL_DIRECT, F.FOE_MODEL_ANS_L2])
def test_tc_gradient(dev, ctx, bank32, shape, bc, model, prec):
    H, W = shape
    y = synth.poisson_observation(synth.clean_image(H, W, 40 + H), 6.0, 41 + W)
    d = y if model == F.FOE_MODEL_DIRECT else O.anscombe(y)
    rng = np.random.default_rng(H + 3 * W)
    u = (d + rng.uniform(-0.5, 0.5, d.shape)).clip(0.1).astype(F32).astype(np.float64)
    d32 = d.astype(F32).astype(np.float64)
    _, g_ref = problem(bank32, H, W, model, bc, 1e-3).energy_grad(u, d32)
    ud, dd = to_dev(u, dev), to_dev(d32, dev)
    gd = torch.zeros_like(ud)
    F.foe_energy_grad(ctx, ud, dd, H, W, ud.shape[1], model, LAM, bc, prec, grad=gd, energy=False)
    g = from_dev(gd, W)
    scale = np.abs(g_ref).max()
    err = np.abs(g - g_ref).max() / scale
    rms = np.sqrt(((g - g_ref) ** 2).mean()) / np.sqrt((g_ref ** 2).mean())
    print(f"tc grad prec={prec} {shape} bc={bc} model={model}: max rel {err:.2e} rms rel {rms:.2e}")
    # BF16 operands: 8-bit mantissa; TF32: 10-bit mantissa (errors about 4x smaller)
    assert err <= (2e-2 if prec == BF16 else 5e-3) and rms <= (5e-3 if prec == BF16 else 1.5e-3)


@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("shape", [(64, 64), (37, 70), (7, 7), (30, 54), (245, 61), (60, 59), (150, 130), (3335, 60),
                                   (67, 3000), (456, 456)])
@pytest.mark.parametrize("model", [F.FOE_MODEL_DIRECT, F.FOE_MODEL_ANS_L2, F.FOE_MODEL_ANS_IDIV])
def test_tc_single_step(dev, ctx, bank32, shape, model, prec):
    H, W = shape
    bc = F.FOE_BC_SYMMETRIC
    tau, _ = F.foe_step_size(ctx, bc, GAMMA)
    y = synth.poisson_observation(synth.clean_image(H, W, 60 + H), 6.0, 61 + W)
    d = y if model == F.FOE_MODEL_DIRECT else O.anscombe(y)
    rng = np.random.default_rng(H * W + 1)
    u = (d + rng.uniform(-0.3, 0.3, d.shape)).clip(0.05).astype(F32).astype(np.float64)
    delta = rng.uniform(-0.05, 0.05, d.shape).astype(F32).astype(np.float64)
    d32 = d.astype(F32).astype(np.float64)
    pr = problem(bank32, H, W, model, bc, tau)
    ref = pr.step(d32, u, u - delta)
    _, g_ref = pr.energy_grad(u, d32)
    uh, dl, dd = to_dev(u, dev), to_dev(delta, dev), to_dev(d32, dev)
    ul, un = torch.zeros_like(uh), torch.zeros_like(uh)
    F.foe_ipiano_step(ctx, uh, ul, dl, dd, un, H, W, uh.shape[1], model, LAM, tau, GAMMA, bc, prec)
    torch.cuda.synchronize()
    got = from_dev(un, W) + from_dev(ul, W)
    assert np.abs(got - ref).max() <= tau * 2e-2 * np.abs(g_ref).max()


@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("model,peak", [(F.FOE_MODEL_ANS_L2, 4.0), (F.FOE_MODEL_DIRECT, 4.0),
                                        (F.FOE_MODEL_ANS_IDIV, 2.0), (F.FOE_MODEL_AUTO, 8.0)])
def test_tc_denoise_64x64_psnr(dev, ctx, bank32, model, peak, prec):
    H = W = 64
    clean = synth.clean_image(H, W, 1000) * peak
    y = synth.poisson_observation(clean / peak, peak, 5000)
    tau, _ = F.foe_step_size(ctx, F.FOE_BC_SYMMETRIC, GAMMA)
    yd = to_dev(y, dev)
    xd = torch.zeros_like(yd)
    F.foe_denoise(ctx, yd, xd, H, W, yd.shape[1], peak, F.SolveOpts(model=model, iters=100, prec=prec, tau=tau))
    x = from_dev(xd, W)
    ref, _ = problem(bank32, H, W, model, F.FOE_BC_SYMMETRIC, tau).denoise(y, peak, 100)
    dp = abs(O.psnr(x, clean, peak) - O.psnr(ref, clean, peak))
    print(f"tc 64x64 prec={prec} model={model} peak={peak}: dPSNR {dp:.4f} dB, PSNR(x vs oracle) {O.psnr(x, ref, peak):.1f} dB")
    assert dp <= 0.02


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("case", range(15))
def test_tc_512_psnr_vs_oracle(dev, ctx, bank32, case):
    """The benchmark set: 512x512, 300 iterations, peaks {1,2,4,8,30} x {direct, Anscombe-L2, Anscombe-I-divergence}.

    Oracle values come from tests/golden/make_oracle_512.py (oracle only); if the generator no
    longer reproduces the stored inputs the oracle is rerun here.  Bars: PSNR within 0.02 dB of the oracle's for
    BF16 and TF32 (the metric's bar); sampled max-abs on the [0, 255] scale <= 1e-4 for FP32 and <= 1 grey level
    for BF16, about twice the largest BF16 figure measured on this set (0.55, direct model at peak 30), so that a
    localised artefact cannot hide inside a PSNR average."""
    g = _golden()
    c = g["cases"][case]
    H, W, peak, model = g["H"], g["W"], c["peak"], c["model"]
    pi = [1.0, 2.0, 4.0, 8.0, 30.0].index(peak)
    seed = 1000 + 10 * pi
    clean = synth.clean_image(H, W, seed) * peak
    y = synth.poisson_observation(clean / peak, peak, seed + 5000)
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(os.path.dirname(GOLDEN), "make_oracle_512.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    k32, a32 = bank32
    if mk.input_hash(k32, a32, y) == c["input_hash"]:
        psnr_ref = c["psnr_oracle"]
        xs_ref = np.array(c["x_sample"])
    else:
        ref, _ = problem(bank32, H, W, model, F.FOE_BC_SYMMETRIC, g["tau"]).denoise(y, peak, g["iters"])
        psnr_ref = O.psnr(ref, clean, peak)
        xs_ref = ref.ravel()[np.array(g["sample_index"])]
    yd = to_dev(y, dev)
    out = {}
    for prec in (BF16, TF32, F.FOE_PREC_FP32):
        xd = torch.zeros_like(yd)
        F.foe_denoise(ctx, yd, xd, H, W, yd.shape[1], peak,
                      F.SolveOpts(model=model, iters=g["iters"], prec=prec, tau=g["tau"], gamma=GAMMA))
        out[prec] = from_dev(xd, W)
    dp = abs(O.psnr(out[BF16], clean, peak) - psnr_ref)
    dp32 = abs(O.psnr(out[TF32], clean, peak) - psnr_ref)
    xs32 = out[F.FOE_PREC_FP32].ravel()[np.array(g["sample_index"])]
    err32 = np.abs(xs32 - xs_ref).max() * 255.0 / peak
    errbf = np.abs(out[BF16].ravel()[np.array(g["sample_index"])] - xs_ref).max() * 255.0 / peak
    print(f"512 {c['name']} peak {peak}: dPSNR(bf16) {dp:.4f} dB, dPSNR(tf32) {dp32:.4f} dB; "
          f"sampled max-abs fp32 {err32:.2e}, bf16 {errbf:.2e}")
    assert dp <= 0.02 and dp32 <= 0.02
    assert err32 <= 1e-4
    assert errbf <= 1.0
