"""The stopping rule on the GPU: ||u^n - u^{n-1}|| <= tol ||u^n|| checked every tol_every steps in FP64.

The paper reports iteration counts to convergence (Sec. 5.1) without fixing a rule; the oracle's reading of it
(orc_ipiano_tol) is pinned in test_oracle_pins.py.  Here:
  * plain FP32: the same stopping step as the oracle, and the output within the whole-solve FP32 bound
    (max-abs <= 1e-4 on the [0, 255] scale).  The tolerance is placed between two checks of the oracle's own
    trajectory with a 5 % margin each side, so that FP32 rounding cannot move the decision;
  * every precision and entry point: the output after a stop at n is bitwise the fixed-budget solve of n steps
    (the step kernels are deterministic), which checks that launches past the stop leave the image alone and
    that the output map reads the plane of n's parity (odd and even n both occur);
  * batches: per-image counts, and images whose budget ends before their stop.
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


def to_dev(a, dev):
    a = np.asarray(a, dtype=F32)
    H, W = a.shape
    t = torch.zeros((H, ld_of(W)), dtype=torch.float32, device=dev)
    t[:, :W] = torch.from_numpy(np.ascontiguousarray(a))
    return t


def solve(dev, ctx, y, peak, opts, static=False):
    H, W = y.shape
    yd = to_dev(y, dev)
    xd = torch.zeros_like(yd)
    if static:
        F.foe_denoise_static(ctx, yd, xd, H, W, yd.shape[1], peak, opts)
        rep = {"iters_done": F.foe_iters_done(ctx, 1)[0]}
    else:
        rep = F.foe_denoise(ctx, yd, xd, H, W, yd.shape[1], peak, opts, report=True)
        assert F.foe_iters_done(ctx, 1)[0] == rep["iters_done"]
    torch.cuda.synchronize()
    return xd[:, :W].cpu().numpy(), rep


def oracle_checks(bank32, y, model, tau, iters, every):
    """Relative changes of the oracle's iterate at the checks n = every, 2 every, ... (model resolved)."""
    H, W = y.shape
    k, a = bank32
    pr = O.Problem(k.astype(np.float64), a.astype(np.float64), H, W, model=model, lam=1.0, tau=tau, gamma=GAMMA)
    d = y if model == O.MODEL_DIRECT else O.anscombe(y)
    u, up = d.copy(), d.copy()
    out = {}
    for n in range(1, iters + 1):
        up, u = u, pr.step(d, u, up)
        if n % every == 0:
            out[n] = float(np.linalg.norm(u - up) / np.linalg.norm(u))
    return pr, out


def separated_tol(ratios, n_min):
    """(m, tol): a tolerance whose first success is the check at m >= n_min, 5 % from the ratio there and from the
    smallest ratio of every earlier check."""
    ns = sorted(ratios)
    for i, n in enumerate(ns):
        if n < n_min or i == 0:
            continue
        tol = ratios[n] * 1.05
        if min(ratios[k] for k in ns[:i]) > tol * 1.05:
            return n, tol
    raise AssertionError("no separated check")


@pytest.mark.parametrize("model,peak,every", [(F.FOE_MODEL_ANS_L2, 8.0, 10), (F.FOE_MODEL_ANS_IDIV, 2.0, 7),
                                              (F.FOE_MODEL_DIRECT, 6.0, 9)])
def test_fp32_stops_where_the_oracle_stops(dev, ctx, bank32, model, peak, every):
    H, W = 64, 70
    y = synth.poisson_observation(synth.clean_image(H, W, 1000), peak, 5000)
    tau, _ = F.foe_step_size(ctx, F.FOE_BC_SYMMETRIC, GAMMA)
    pr, ratios = oracle_checks(bank32, y, model, tau, 200, every)
    m, tol = separated_tol(ratios, 60)
    ref, _, n_ref = pr.denoise_tol(y, peak, 200, float(F32(tol)), every)
    assert n_ref == m
    opts = F.SolveOpts(model=model, iters=200, prec=F.FOE_PREC_FP32, tau=tau, tol=tol, tol_every=every)
    x, rep = solve(dev, ctx, y, peak, opts)
    assert rep["iters_done"] == m
    assert np.abs(x - ref).max() * 255.0 / peak <= 1e-4


@pytest.mark.parametrize("prec,shape", [(F.FOE_PREC_BF16, (480, 450)), (F.FOE_PREC_BF16, (40, 50)),
                                        (F.FOE_PREC_TF32, (70, 64)), (F.FOE_PREC_FP32, (33, 47))])
@pytest.mark.parametrize("every", [10, 7])
def test_stop_equals_the_fixed_budget_solve_of_that_length(dev, ctx, prec, shape, every):
    H, W = shape
    y = synth.poisson_observation(synth.clean_image(H, W, 11 + H), 4.0, 12 + W)
    opts = dict(model=F.FOE_MODEL_AUTO, prec=prec)
    x, rep = solve(dev, ctx, y, 4.0, F.SolveOpts(iters=300, tol=1e-3, tol_every=every, **opts))
    n = rep["iters_done"]
    assert 0 < n < 300 and n % every == 0
    x_ref, rep_ref = solve(dev, ctx, y, 4.0, F.SolveOpts(iters=n, **opts))
    assert rep_ref["iters_done"] == n
    assert np.array_equal(x, x_ref)
    # the static entry point takes the same decisions
    xs, reps = solve(dev, ctx, y, 4.0, F.SolveOpts(iters=300, tol=1e-3, tol_every=every, **opts), static=True)
    assert reps["iters_done"] == n and np.array_equal(xs, x)


def test_budget_before_the_stop_and_tol_zero(dev, ctx):
    y = synth.poisson_observation(synth.clean_image(64, 64, 3), 4.0, 4)
    x, rep = solve(dev, ctx, y, 4.0, F.SolveOpts(iters=25, tol=1e-6, tol_every=10))
    assert rep["iters_done"] == 25
    x_ref, rep_ref = solve(dev, ctx, y, 4.0, F.SolveOpts(iters=25))
    assert rep_ref["iters_done"] == 25 and np.array_equal(x, x_ref)


@pytest.mark.parametrize("graph", [False, True])
def test_batch_per_image_counts(dev, ctx, graph):
    shapes = [(450, 460, 300), (64, 90, 300), (40, 33, 300), (130, 70, 30), (96, 200, 300)]
    ys, xs, descs = [], [], []
    for j, (H, W, iters) in enumerate(shapes):
        y = to_dev(synth.poisson_observation(synth.clean_image(H, W, 50 + j), 3.0 + j, 60 + j), dev)
        ys.append(y)
        xs.append(torch.zeros_like(y))
        descs.append({"y": y, "x": xs[-1], "H": H, "W": W, "ld": y.shape[1], "peak": 3.0 + j, "iters": iters})
    opts = dict(model=F.FOE_MODEL_AUTO, prec=F.FOE_PREC_BF16)
    stream = torch.cuda.Stream() if graph else None
    F.foe_denoise_batch(ctx, descs, F.SolveOpts(tol=1e-3, tol_every=10, use_graph=graph, **opts),
                        stream=stream.cuda_stream if graph else None)
    done = F.foe_iters_done(ctx, len(descs), stream=stream.cuda_stream if graph else None)
    torch.cuda.synchronize()
    assert done[3] == 30                                   # its budget ends before its stop
    assert all(0 < n < 300 and n % 10 == 0 for j, n in enumerate(done) if j != 3)
    for j, (H, W, _) in enumerate(shapes):
        single = torch.zeros_like(ys[j])
        F.foe_denoise(ctx, ys[j], single, H, W, ys[j].shape[1], descs[j]["peak"], F.SolveOpts(iters=done[j], **opts))
        torch.cuda.synchronize()
        assert torch.equal(single[:, :W], xs[j][:, :W]), j


def test_backtracking_with_the_stopping_rule(dev, ctx):
    y = synth.poisson_observation(synth.clean_image(48, 40, 21), 6.0, 22)
    opts = dict(model=F.FOE_MODEL_ANS_L2, prec=F.FOE_PREC_FP32, step=F.FOE_STEP_BACKTRACK)
    x, rep = solve(dev, ctx, y, 6.0, F.SolveOpts(iters=200, tol=3e-4, tol_every=5, **opts))
    n = rep["iters_done"]
    assert 0 < n < 200 and n % 5 == 0
    x_ref, _ = solve(dev, ctx, y, 6.0, F.SolveOpts(iters=n, **opts))
    assert np.array_equal(x, x_ref)


def test_invalid_stopping_options(dev, ctx, bank32):
    y = to_dev(np.ones((16, 16)), dev)
    x = torch.zeros_like(y)
    for kw in (dict(tol=-1.0), dict(tol=float("nan")), dict(tol=1e-3, tol_every=0)):
        with pytest.raises(F.FoeError) as e:
            F.foe_denoise(ctx, y, x, 16, 16, 16, 4.0, F.SolveOpts(**kw))
        assert e.value.status == F.FOE_EINVAL
    with pytest.raises(F.FoeError) as e:
        F.foe_iters_done(ctx, 3)
    assert e.value.status == F.FOE_EINVAL
    with pytest.raises(F.FoeError) as e:
        F.foe_server_create(ctx, 1 << 24, 4, 5, False, F.SolveOpts(tol=1e-3))
    assert e.value.status == F.FOE_EUNSUPPORTED
