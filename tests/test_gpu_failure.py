"""Failure detection and checkpoint / resume on the device, without faulting the GPU.

Every wait of the tensor-core kernel is bounded: a test makes one CTA withhold one mbarrier arrival
(foe_debug_withhold_arrival), so that its waits expire after about 2 s; the call must report FOE_ETIMEOUT and the
context must stay usable.  Nothing traps, faults or spins without limit.  Checkpoint / resume: a step-driven solve
(foe_ipiano_step) whose state is copied to the host after n steps and restored into fresh buffers continues
bit for bit as the uninterrupted run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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
    c = F.foe_create(k, a)
    yield c
    F.foe_destroy(c)


def _image(H, W, seed):
    y = synth.poisson_observation(synth.clean_image(H, W, seed), 4.0, seed + 1)
    return torch.from_numpy(y.astype(np.float32)).cuda()


@pytest.mark.parametrize("side", [64, 456])   # the 26 x 26 kernel, the pixel-pair kernel
def test_an_expired_device_wait_is_reported_and_the_context_recovers(ctx, side):
    H = W = side
    y = _image(H, W, 31)
    opts = F.SolveOpts(model=F.FOE_MODEL_ANS_L2, prec=F.FOE_PREC_BF16, iters=10)
    ref = torch.zeros_like(y)
    F.foe_denoise(ctx, y, ref, H, W, W, 4.0, opts, report=True)
    # with a report: the call raises FOE_ETIMEOUT and clears the status
    F.foe_debug_withhold_arrival(ctx)
    x = torch.zeros_like(y)
    with pytest.raises(F.FoeError) as e:
        F.foe_denoise(ctx, y, x, H, W, W, 4.0, opts, report=True)
    assert e.value.status == F.FOE_ETIMEOUT
    assert F.foe_device_status(ctx) == F.FOE_OK
    # without a report: the status stays until foe_device_status reads and clears it
    F.foe_debug_withhold_arrival(ctx)
    F.foe_denoise(ctx, y, x, H, W, W, 4.0, opts)
    assert F.foe_device_status(ctx) == F.FOE_ETIMEOUT
    assert F.foe_device_status(ctx) == F.FOE_OK
    # the context is usable again and computes what it computed before
    F.foe_denoise(ctx, y, x, H, W, W, 4.0, opts, report=True)
    torch.cuda.synchronize()
    assert torch.equal(x, ref)


@pytest.mark.parametrize("prec", [F.FOE_PREC_FP32, F.FOE_PREC_BF16])
def test_resume_from_a_host_checkpoint_is_bitwise_identical(ctx, prec, tmp_path):
    H, W, n = 300, 700, 12   # 210000 pixels: the pixel-pair kernel's 58 x 58 tiles on the BF16 path
    ld = (W + 3) // 4 * 4
    y = synth.poisson_observation(synth.clean_image(H, W, 41), 4.0, 42)
    v = 2.0 * np.sqrt(y + 3.0 / 8.0)
    d = torch.zeros((H, ld), dtype=torch.float32, device="cuda")
    d[:, :W] = torch.from_numpy(v.astype(np.float32))
    tau, _ = F.foe_step_size(ctx, F.FOE_BC_SYMMETRIC, 0.8)

    def fresh():
        return d.clone(), torch.zeros_like(d), torch.zeros_like(d)   # u_hi, u_lo, delta

    def steps(state, k):
        uh, ul, dl = state
        for _ in range(k):
            un = torch.empty_like(uh)
            F.foe_ipiano_step(ctx, uh, ul, dl, d, un, H, W, ld, F.FOE_MODEL_ANS_L2, 1.0, tau, 0.8,
                              F.FOE_BC_SYMMETRIC, prec)
            uh = un
        return uh, ul, dl

    straight = steps(fresh(), 2 * n)
    half = steps(fresh(), n)
    torch.cuda.synchronize()
    path = tmp_path / "state.npz"
    np.savez(path, *[t.cpu().numpy() for t in half])
    del half
    loaded = np.load(path)
    resumed = steps(tuple(torch.from_numpy(loaded[f"arr_{i}"]).cuda() for i in range(3)), n)
    torch.cuda.synchronize()
    for a, b in zip(straight, resumed):  # image columns (the pitch padding of fresh outputs is never written)
        assert torch.equal(a[:, :W], b[:, :W])


@pytest.mark.parametrize("prec", [F.FOE_PREC_FP32, F.FOE_PREC_BF16])
def test_non_finite_outputs_are_reported(ctx, prec):
    # a NaN in the data spreads through the responses of its neighbourhood; with a report the call counts the
    # non-finite outputs and returns FOE_ENONFINITE (without one it returns normally)
    H = W = 48
    y = _image(H, W, 51)
    y[20, 20] = float("nan")
    x = torch.zeros_like(y)
    opts = F.SolveOpts(model=F.FOE_MODEL_ANS_L2, prec=prec, iters=3)
    F.foe_denoise(ctx, y, x, H, W, W, 4.0, opts)
    with pytest.raises(F.FoeError) as e:
        F.foe_denoise(ctx, y, x, H, W, W, 4.0, opts, report=True)
    assert e.value.status == F.FOE_ENONFINITE
    assert int((~torch.isfinite(x)).sum()) > 1
    rep = F.foe_denoise(ctx, _image(H, W, 52), x, H, W, W, 4.0, opts, report=True)
    assert rep["nonfinite"] == 0 and F.foe_device_status(ctx) == F.FOE_OK
