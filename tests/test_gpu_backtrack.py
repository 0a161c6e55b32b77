"""Step control by Lipschitz backtracking (FOE_STEP_BACKTRACK, FP32 path) against the FP64 oracle.

Accept / reject decisions compare FP64 sums of FP32-evaluated energies, so a trial whose margin is at rounding
level may be decided differently on the two sides; the oracle therefore replays the GPU's logged step sizes
(the accepted trial of every iteration) and the results are compared at the FP32 path's bar (max-abs 1e-4 on the
255 scale).  Every logged decision is also checked in FP64 on the replayed iterates wherever its margin is above
rounding level.
"""
import math

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
C2 = 2e-3 / 2


@pytest.fixture(scope="module")
def ctx(bank):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    torch.cuda.set_device(0)
    k, a = bank
    c = F.foe_create(k.astype(F32), a.astype(F32))
    yield c
    F.foe_destroy(c)


def _run(ctx, y, peak, model, iters, tau_seed=0.0):
    H, W = y.shape
    ld = (W + 3) // 4 * 4
    yd = torch.zeros((H, ld), dtype=torch.float32, device="cuda")
    yd[:, :W] = torch.from_numpy(y.astype(F32))
    xd = torch.zeros_like(yd)
    rep = F.foe_denoise(ctx, yd, xd, H, W, ld, peak,
                        F.SolveOpts(model=model, iters=iters, prec=F.FOE_PREC_FP32, step=F.FOE_STEP_BACKTRACK,
                                    gamma=GAMMA, tau=tau_seed), report=True)
    tau, acc = F.foe_step_log(ctx)
    return xd[:, :W].double().cpu().numpy(), rep, tau, acc


def _replay(bank, y, peak, model, taus):
    """The oracle's iPiano driven by the given step sizes (one per iteration), then the output map."""
    k, a = bank
    H, W = y.shape
    d = y.astype(np.float64) if model == F.FOE_MODEL_DIRECT else O.anscombe(y)
    pr = O.Problem(k.astype(F32).astype(np.float64), a.astype(F32).astype(np.float64), H, W, model=model,
                   lam=1.0, gamma=GAMMA)
    u, up = d.copy(), d.copy()
    states = [(u, up)]
    for t in taus:
        un = pr.step(d, u, up, tau=float(t))
        up, u = u, un
        states.append((u, up))
    x = u if model == F.FOE_MODEL_DIRECT else O.inverse(np.maximum(u, math.sqrt(1.5)))
    return x, states, pr, d


@pytest.mark.parametrize("model,peak,shape", [(F.FOE_MODEL_ANS_L2, 4.0, (64, 64)), (F.FOE_MODEL_DIRECT, 2.0, (48, 70)),
                                              (F.FOE_MODEL_ANS_IDIV, 3.0, (37, 53))])
def test_backtracking_matches_oracle_replay(ctx, bank, model, peak, shape):
    H, W = shape
    iters = 60
    clean = synth.clean_image(H, W, 300 + H) * peak
    y = synth.poisson_observation(clean / peak, peak, 301 + W)
    x, rep, tau, acc = _run(ctx, y, peak, model, iters)
    assert rep["iters_done"] == iters and acc.sum() == iters
    assert rep["backtracks"] == int((~acc).sum())
    # the log follows the rule: L = 2 (1 - gamma) / tau - 2 c2 doubles after a rejection, shrinks by 1.5 after
    # an acceptance
    L = 2 * (1 - GAMMA) / tau.astype(np.float64) - 2 * C2
    for i in range(len(L) - 1):
        want = L[i] * 2.0 if not acc[i] else L[i] / 1.5
        assert math.isclose(L[i + 1], want, rel_tol=2e-5)
    taus = tau[acc]
    xr, states, pr, d = _replay(bank, y, peak, model, taus)
    err = np.abs(x - xr).max() * 255.0 / peak
    print(f"backtrack model={model} {shape}: {len(tau)} trials, {int((~acc).sum())} rejected, max-abs {err:.2e}")
    assert err <= 1e-4
    # FP64 check of every logged decision on the replayed iterates (where the margin exceeds rounding level)
    k, a = pr.k, pr.alpha
    it = 0
    for t, ok in zip(tau.astype(np.float64), acc):
        u, up = states[it]
        Fu = O.prior_energy(k, a, u)
        g = O.prior_grad(k, a, u)
        un = pr.step(d, u, up, tau=t)
        du = un - u
        Lt = 2 * (1 - GAMMA) / t - 2 * C2
        margin = Fu + float(np.sum(g * du)) + 0.5 * Lt * float(np.sum(du * du)) - O.prior_energy(k, a, un)
        if abs(margin) > 1e-5 * abs(Fu):
            assert (margin >= 0) == bool(ok), (it, margin)
        if ok:
            it += 1


def test_backtracking_from_a_small_seed_rejects_then_recovers(ctx, bank):
    # tau_seed far above 2 (1 - gamma) / L^: the first trials are rejected, L doubles until the test passes
    H = W = 40
    peak = 4.0
    y = synth.poisson_observation(synth.clean_image(H, W, 77), peak, 78)
    tau_fixed, Lhat = F.foe_step_size(ctx, F.FOE_BC_SYMMETRIC, GAMMA)
    x, rep, tau, acc = _run(ctx, y, peak, F.FOE_MODEL_ANS_L2, 20, tau_seed=tau_fixed * 400.0)
    assert rep["backtracks"] >= 5 and not acc[0]
    xr, *_ = _replay(bank, y, peak, F.FOE_MODEL_ANS_L2, tau[acc])
    assert np.abs(x - xr).max() * 255.0 / peak <= 1e-4


def test_backtracking_is_fp32_and_single_image_only(ctx):
    y = torch.ones((16, 16), device="cuda")
    x = torch.zeros_like(y)
    with pytest.raises(F.FoeError) as e:
        F.foe_denoise(ctx, y, x, 16, 16, 16, 4.0, F.SolveOpts(step=F.FOE_STEP_BACKTRACK, prec=F.FOE_PREC_BF16))
    assert e.value.status == F.FOE_EUNSUPPORTED
    with pytest.raises(F.FoeError) as e:
        F.foe_denoise_batch(ctx, [{"y": y, "x": x, "H": 16, "W": 16, "ld": 16, "peak": 4.0, "iters": 5}],
                            F.SolveOpts(step=F.FOE_STEP_BACKTRACK, prec=F.FOE_PREC_FP32))
    assert e.value.status == F.FOE_EUNSUPPORTED
