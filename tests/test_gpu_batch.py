"""Batched uneven instances in one graph: 64 images, sides from {128, ..., 1024} (H and W drawn
independently), peaks log-uniform in [1, 30], per-image budgets of 100-300 iterations, BF16.

At this size the oracle is checked image by image through foe_denoise (itself checked against the
oracle at 512x512 and on small images): every image of the graph-captured batch must equal its own
single-image solve bit for bit, as the batched kernel computes each tile from the same inputs.  A
small batch is also compared with the oracle directly.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1609_05722_gb300 import build as B  # noqa: E402
from paper_1609_05722_gb300 import foe as F  # noqa: E402
from paper_1609_05722_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    torch.cuda.set_device(0)
    k, a = synth.filter_bank()
    c = F.foe_create(k.astype(np.float32), a.astype(np.float32))
    yield c
    F.foe_destroy(c)


def upload(specs):
    ys, xs, descs = [], [], []
    for s in specs:
        _, y = synth.make_problem(s)
        ld = (s.W + 3) // 4 * 4
        yd = torch.zeros((s.H, ld), dtype=torch.float32, device="cuda")
        yd[:, :s.W] = torch.from_numpy(y.astype(np.float32)).cuda()
        xd = torch.zeros_like(yd)
        ys.append(yd)
        xs.append(xd)
        descs.append({"y": yd, "x": xd, "H": s.H, "W": s.W, "ld": ld, "peak": s.peak, "iters": s.iters})
    return ys, xs, descs


def test_graph_batch_of_64_equals_single_solves(ctx):
    specs = synth.batched_uneven_specs(64, seed=3)
    ys, xs, descs = upload(specs)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        opts = F.SolveOpts(model=F.FOE_MODEL_AUTO, prec=F.FOE_PREC_BF16, use_graph=True)
        F.foe_denoise_batch(ctx, descs, opts, stream=stream)
        first = [x.clone() for x in xs]
        for x in xs:
            x.zero_()
        F.foe_denoise_batch(ctx, descs, opts, stream=stream)  # replays the cached graph
    stream.synchronize()
    for j, s in enumerate(specs):
        assert torch.equal(first[j], xs[j]), j
        single = torch.zeros_like(xs[j])
        F.foe_denoise(ctx, ys[j], single, s.H, s.W, descs[j]["ld"], s.peak,
                      F.SolveOpts(model=F.FOE_MODEL_AUTO, prec=F.FOE_PREC_BF16, iters=s.iters))
        torch.cuda.synchronize()
        assert torch.equal(single[:, :s.W], xs[j][:, :s.W]), j


@pytest.mark.parametrize("prec", [F.FOE_PREC_FP32, F.FOE_PREC_BF16])
def test_small_graph_batch_against_oracle(ctx, prec):
    specs = [synth.ImageSpec(40, 72, 2.0, 30, 11, 12), synth.ImageSpec(96, 33, 9.0, 45, 13, 14),
             synth.ImageSpec(64, 64, 30.0, 12, 15, 16), synth.ImageSpec(17, 130, 1.0, 0, 17, 18)]
    ys, xs, descs = upload(specs)
    stream = torch.cuda.Stream()
    tau, _ = F.foe_step_size(ctx, F.FOE_BC_SYMMETRIC, float(np.float32(0.8)))
    with torch.cuda.stream(stream):
        F.foe_denoise_batch(ctx, descs, F.SolveOpts(model=F.FOE_MODEL_AUTO, prec=prec, tau=tau, use_graph=True),
                            stream=stream)
    stream.synchronize()
    k, a = synth.filter_bank()
    for j, s in enumerate(specs):
        clean, y = synth.make_problem(s)
        pr = O.Problem(k.astype(np.float32).astype(np.float64), a.astype(np.float32).astype(np.float64), s.H, s.W,
                       model=O.MODEL_AUTO, lam=1.0, tau=tau, gamma=float(np.float32(0.8)))
        ref, _ = pr.denoise(y, s.peak, s.iters)
        x = xs[j][:, :s.W].double().cpu().numpy()
        if prec == F.FOE_PREC_FP32:
            assert np.abs(x - ref).max() * 255.0 / s.peak <= 1e-4
        else:
            assert abs(O.psnr(x, clean, s.peak) - O.psnr(ref, clean, s.peak)) <= 0.02


@pytest.mark.parametrize("prec", [F.FOE_PREC_BF16, F.FOE_PREC_TF32])
def test_zero_padding_batch_equals_single_solves(ctx, prec):
    # 8 images of 512 x 256: the batch has several tiles per CTA (the next tile's input region, zero rows
    # included, is prefetched while a tile is computed), a single image at most one per CTA
    specs = [synth.ImageSpec(512, 256, p, 20, 21 + j, 31 + j) for j, p in enumerate([1.0, 2.0, 4.0, 8.0] * 2)]
    ys, xs, descs = upload(specs)
    opts = dict(model=F.FOE_MODEL_AUTO, prec=prec, bc=F.FOE_BC_ZERO)
    F.foe_denoise_batch(ctx, descs, F.SolveOpts(**opts))
    torch.cuda.synchronize()
    for j, s in enumerate(specs):
        single = torch.zeros_like(xs[j])
        F.foe_denoise(ctx, ys[j], single, s.H, s.W, descs[j]["ld"], s.peak, F.SolveOpts(iters=s.iters, **opts))
        torch.cuda.synchronize()
        assert torch.equal(single[:, :s.W], xs[j][:, :s.W]), j


def test_per_image_data_terms_in_one_batch(ctx):
    # one batch, each image with its own data term (use_model = 1) or the batch's (opts.model): every image equals
    # its single solve under that model bit for bit; sizes on both sides of the pixel-pair threshold
    specs = [synth.ImageSpec(512, 512, p, 30, 41 + j, 51 + j) for j, p in enumerate([1.0, 4.0, 8.0])] + \
            [synth.ImageSpec(160, 200, p, 30, 61 + j, 71 + j) for j, p in enumerate([2.0, 30.0, 6.0])]
    models = [F.FOE_MODEL_DIRECT, F.FOE_MODEL_ANS_L2, None, F.FOE_MODEL_ANS_IDIV, F.FOE_MODEL_AUTO, None]
    ys, xs, descs = upload(specs)
    for d, m in zip(descs, models):
        if m is not None:
            d["model"] = m
    F.foe_denoise_batch(ctx, descs, F.SolveOpts(model=F.FOE_MODEL_ANS_L2, prec=F.FOE_PREC_BF16))
    torch.cuda.synchronize()
    for j, (s, m) in enumerate(zip(specs, models)):
        single = torch.zeros_like(xs[j])
        F.foe_denoise(ctx, ys[j], single, s.H, s.W, descs[j]["ld"], s.peak,
                      F.SolveOpts(model=F.FOE_MODEL_ANS_L2 if m is None else m, iters=s.iters, prec=F.FOE_PREC_BF16))
        torch.cuda.synchronize()
        assert torch.equal(single[:, :s.W], xs[j][:, :s.W]), j
    # a model outside the enumeration is refused
    bad = [dict(descs[0], model=7)]
    with pytest.raises(F.FoeError) as e:
        F.foe_denoise_batch(ctx, bad, F.SolveOpts())
    assert e.value.status == F.FOE_EINVAL
