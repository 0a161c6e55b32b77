"""foe_denoise_static: denoising with the library's fixed device workspace, no allocation.

It serves callers that cannot allocate device memory when they call (code whose memory belongs to
another allocator or a fixed arena, real-time loops that cannot absorb the synchronisation of cudaMalloc
and cudaFree).  The test calls it through the C ABI and checks each result against the allocating entry
point foe_denoise, within the plain-FP32 parity tolerance used elsewhere (max-abs 1e-4 on the [0, 255]
scale) and, since both run the same kernels on the same inputs, bit for bit, on two calls in a row with
different images, so that the second call cannot pass by reusing the first call's workspace contents.
This file is collected last; it must pass alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1609_05722_gb300 import build as B  # noqa: E402
from paper_1609_05722_gb300 import foe as F  # noqa: E402
from paper_1609_05722_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _image(H, W, peak, seed, dev):
    ld = (W + 3) // 4 * 4
    y = synth.poisson_observation(synth.clean_image(H, W, seed), peak, seed + 1).astype(np.float32)
    t = torch.zeros((H, ld), dtype=torch.float32, device=dev)
    t[:, :W] = torch.from_numpy(y)
    return t, ld


def test_static_workspace_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    k, a = synth.filter_bank()
    ctx = F.foe_create(k.astype(np.float32), a.astype(np.float32))
    try:
        cases = [(64, 64, 4.0, 11), (131, 200, 12.0, 21)]  # two calls in a row, different shapes
        for prec in (F.FOE_PREC_FP32, F.FOE_PREC_BF16):
            opts = F.SolveOpts(model=F.FOE_MODEL_AUTO, iters=40, prec=prec)
            for H, W, peak, seed in cases:
                y, ld = _image(H, W, peak, seed, dev)
                x_ref = torch.zeros_like(y)
                x_sta = torch.full_like(y, float("nan"))
                F.foe_denoise(ctx, y, x_ref, H, W, ld, peak, opts)
                F.foe_denoise_static(ctx, y, x_sta, H, W, ld, peak, opts)
                torch.cuda.synchronize()
                ref = x_ref[:, :W].double().cpu().numpy()
                got = x_sta[:, :W].double().cpu().numpy()
                assert np.isfinite(got).all()
                assert np.abs(got - ref).max() * 255.0 / peak <= 1e-4
                assert np.array_equal(got, ref)
        # beyond the stated maximum (H * ld > 2**20) the call is refused before any device work
        y, ld = _image(64, 64, 4.0, 5, dev)
        with pytest.raises(F.FoeError) as e:
            F.foe_denoise_static(ctx, y, y, 1025, 1024, 1024, 4.0, F.SolveOpts(iters=1))
        assert e.value.status == F.FOE_EINVAL
        assert "static workspace" in F.foe_last_error(ctx)
    finally:
        F.foe_destroy(ctx)


def test_static_entry_point_shows_an_expired_device_wait_as_nan():
    """A device-side wait that expired earlier in the context leaves a sticky FOE_ETIMEOUT that makes the step
    launches return at once.  The static entry point does not synchronise, so it cannot return that status; its
    output is NaN instead of a stale iterate, and foe_device_status reports (and clears) the status."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    k, a = synth.filter_bank()
    ctx = F.foe_create(k.astype(np.float32), a.astype(np.float32))
    try:
        H, W, peak = 64, 64, 4.0
        y, ld = _image(H, W, peak, 31, dev)
        opts = F.SolveOpts(model=F.FOE_MODEL_AUTO, iters=10, prec=F.FOE_PREC_BF16)
        x_ref = torch.zeros_like(y)
        F.foe_denoise(ctx, y, x_ref, H, W, ld, peak, opts)
        # the next tensor-core launch withholds one arrival, so its bounded wait expires (about 2 s)
        F.foe_debug_withhold_arrival(ctx)
        x = torch.zeros_like(y)
        F.foe_denoise_static(ctx, y, x, H, W, ld, peak, opts)
        torch.cuda.synchronize()
        assert torch.isnan(x[:, :W]).all()
        assert F.foe_device_status(ctx) == F.FOE_ETIMEOUT
        assert F.foe_device_status(ctx) == F.FOE_OK
        # the status is clear again: the same call gives the allocating entry point's result
        F.foe_denoise_static(ctx, y, x, H, W, ld, peak, opts)
        torch.cuda.synchronize()
        assert torch.equal(x[:, :W], x_ref[:, :W])
    finally:
        F.foe_destroy(ctx)
