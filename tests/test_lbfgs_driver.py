"""The L-BFGS outer loop of the prior training (Algorithm 1, Sec. 2.5) on the CPU: the driver is given the FP64
oracle's loss and implicit-differentiation gradient (Eq. implicitdifferentiation) on a small problem, so its
iteration and its three stopping rules are checked without a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1609_05722_gb300 import synth  # noqa: E402
from paper_1609_05722_gb300.train import lbfgs_train  # noqa: E402

H, W, B, T, NF = 8, 9, 2, 400, 6


@pytest.fixture(scope="module")
def problem(bank):
    k, a = bank
    clean = np.stack([synth.clean_image(H, W, 70 + s) * 4.0 for s in range(B)])
    noisy = np.stack([synth.poisson_observation(clean[s] / 4.0, 4.0, 80 + s) for s in range(B)])
    return k[:NF].copy(), a[:NF].copy(), clean, noisy


def make_loss(clean, noisy, calls):
    class OracleLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, kt, lat):
            k = kt.detach().numpy()
            a = np.exp(lat.detach().numpy())
            gamma = 0.8
            tau = 0.99 * 2 * (1 - gamma) / (O.lipschitz(k, a) + 2e-3)
            pr = O.Problem(k, a, H, W, model=O.MODEL_ANS_L2, lam=1.0, tau=tau, gamma=gamma, nthreads=1)
            L, dk, da, _, _ = pr.train_grad_implicit(clean, noisy, T, 500, 1e-10)
            calls.append(L)
            ctx.save_for_backward(torch.from_numpy(dk), torch.from_numpy(da))
            return torch.tensor(L, dtype=torch.float64)

        @staticmethod
        def backward(ctx, g):
            dk, da = ctx.saved_tensors
            return g * dk, g * da

    return OracleLoss.apply


def test_lbfgs_decreases_the_loss_and_stops_on_the_iteration_budget(problem):
    k, a, clean, noisy = problem
    calls = []
    kt, lat, losses, reason = lbfgs_train(make_loss(clean, noisy, calls), torch.from_numpy(k).double(),
                                          torch.from_numpy(np.log(a)).double(), max_iter=4, tol=0.0)
    assert reason == "max_iter" and len(losses) == 5
    assert all(l1 < l0 for l0, l1 in zip(losses, losses[1:]))
    assert losses[-1] < 0.98 * losses[0]
    assert kt.shape == (NF, 7, 7) and lat.shape == (NF,)


def test_lbfgs_stops_on_the_relative_change(problem):
    k, a, clean, noisy = problem
    kt, lat, losses, reason = lbfgs_train(make_loss(clean, noisy, []), torch.from_numpy(k).double(),
                                          torch.from_numpy(np.log(a)).double(), max_iter=50, tol=5e-2)
    assert reason == "tol"
    assert abs(losses[-2] - losses[-1]) <= 5e-2 * abs(losses[-2])
    assert all(abs(l0 - l1) > 5e-2 * abs(l0) for l0, l1 in zip(losses[:-2], losses[1:-1]))


def test_lbfgs_stops_when_no_step_decreases_the_loss():
    # a loss with a constant value and a non-zero gradient: the line search cannot decrease it
    class Flat(torch.autograd.Function):
        @staticmethod
        def forward(ctx, kt, lat):
            return torch.tensor(1.0, dtype=torch.float64)

        @staticmethod
        def backward(ctx, g):
            return torch.ones(6, 7, 7, dtype=torch.float64) * g, torch.ones(6, dtype=torch.float64) * g

    _, _, losses, reason = lbfgs_train(Flat.apply, torch.zeros(6, 7, 7, dtype=torch.float64),
                                       torch.zeros(6, dtype=torch.float64), max_iter=10, tol=0.0)
    assert reason == "no_decrease" and len(losses) == 2


def test_lbfgs_resumes_from_a_checkpoint_bit_for_bit(problem, tmp_path):
    k, a, clean, noisy = problem
    k0, la0 = torch.from_numpy(k).double(), torch.from_numpy(np.log(a)).double()
    straight = lbfgs_train(make_loss(clean, noisy, []), k0, la0, max_iter=4, tol=0.0)
    ck = str(tmp_path / "train.pt")
    first = lbfgs_train(make_loss(clean, noisy, []), k0, la0, max_iter=2, tol=0.0, checkpoint=ck)
    assert len(first[2]) == 3
    # a fresh process would start from the same templates; the file holds the parameters and the L-BFGS history
    resumed = lbfgs_train(make_loss(clean, noisy, []), torch.zeros_like(k0), torch.zeros_like(la0), max_iter=4,
                          tol=0.0, checkpoint=ck)
    assert torch.equal(resumed[0], straight[0]) and torch.equal(resumed[1], straight[1])
    assert resumed[2] == straight[2] and resumed[3] == straight[3]


def test_lbfgs_resumed_after_it_stopped_returns_the_stored_result(problem, tmp_path):
    k, a, clean, noisy = problem
    k0, la0 = torch.from_numpy(k).double(), torch.from_numpy(np.log(a)).double()
    ck = str(tmp_path / "stopped.pt")
    done = lbfgs_train(make_loss(clean, noisy, []), k0, la0, max_iter=50, tol=5e-2, checkpoint=ck)
    assert done[3] == "tol"
    # resuming the finished run takes no step and evaluates no loss
    calls = []
    again = lbfgs_train(make_loss(clean, noisy, calls), torch.zeros_like(k0), torch.zeros_like(la0), max_iter=50,
                        tol=5e-2, checkpoint=ck)
    assert calls == []
    assert torch.equal(again[0], done[0]) and torch.equal(again[1], done[1])
    assert again[2] == done[2] and again[3] == "tol"
    # a checkpoint that holds no stopping decision has the criteria re-checked on its last two losses
    st = torch.load(ck, weights_only=False)
    del st["reason"]
    torch.save(st, ck)
    calls = []
    old = lbfgs_train(make_loss(clean, noisy, calls), torch.zeros_like(k0), torch.zeros_like(la0), max_iter=50,
                      tol=5e-2, checkpoint=ck)
    assert calls == [] and old[3] == "tol" and old[2] == done[2]
