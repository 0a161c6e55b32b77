"""Pins of the FP64 oracle against facts fixed outside it.

Each test ties one oracle function to something the oracle does not compute itself: a value
the paper states, a closed form, a library routine on a special case, an exact identity,
a brute-force minimisation or finite differences.  A dropped term, a flipped sign, a
transposed operand or a wrong index in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import optimize, signal
from scipy.stats import poisson

import oracle as O
from paper_1609_05722_gb300 import synth

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(f"{GOLDEN}/{name}") as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                key, val = line.split("=")
                vals[key.strip()] = float(val)
    return vals


# ----------------------------------------------------------------- transforms (Sec. 2.2, 3.1.1)

def test_anscombe_zero_count_value_from_paper():
    # Sec. 3.1.1: a zero count becomes sqrt(3/2) after the Anscombe transform.
    g = _golden("paper_values.txt")
    assert O.anscombe(np.array([0.0]))[0] == pytest.approx(g["anscombe_of_zero"], abs=1e-15)


def test_inverse_anscombe_vanishes_at_zero_count_image():
    # The inverse maps the transform of a zero count back to zero: I_C(sqrt(3/2)) = 0 exactly
    # (3/8 + 1/4 - 11/12 + 5/12 - 1/8 = 0), so the clamp in Eq. FOEscheme's output keeps x >= 0.
    assert abs(O.ic(math.sqrt(1.5))) < 1e-15
    x = O.inverse(np.array([0.1, 1.0, math.sqrt(1.5)]))
    assert np.all(x == 0.0) or abs(x).max() < 1e-15


@pytest.mark.parametrize("lam", [0.1, 0.5, 1.0, 2.0, 4.0, 8.0, 30.0])
def test_inverse_is_nearly_unbiased(lam):
    # Eq. invAns approximates the exact unbiased inverse: I_C(E[2 sqrt(Y + 3/8)]) ~ lambda for
    # Y ~ Poisson(lambda).  The expectation is summed from the pmf; 0.02 guards the closed form's
    # approximation error (every one of its five terms matters at low counts).
    ks = np.arange(0, int(lam * 10 + 80))
    ea = float((poisson.pmf(ks, lam) * O.anscombe(ks.astype(float))).sum())
    assert abs(O.ic(ea) - lam) < 0.02


@pytest.mark.parametrize("z", [1.3, 2.0, 3.0, 7.5])
def test_inverse_derivative_matches_finite_differences(z):
    h = 1e-5
    fd = (O.ic(z + h) - O.ic(z - h)) / (2 * h)
    assert O.ic_deriv(z) == pytest.approx(fd, rel=1e-8, abs=1e-9)


def test_inverse_large_count_asymptote():
    # For large counts E[2 sqrt(Y + 3/8)] ~ 2 sqrt(lambda + 1/8) (Anscombe's expansion), so an
    # unbiased inverse must approach z^2/4 - 1/8.
    for z in (1e3, 1e4):
        assert O.ic(z) - z * z / 4 == pytest.approx(-0.125, abs=1e-3)


# ----------------------------------------------------------------- potential (Eq. STfunc)

@pytest.mark.parametrize("z", [-3.0, -0.7, 0.0, 0.4, 1.0, 2.5, 10.0])
def test_rho_derivatives_match_finite_differences(z):
    h = 1e-5
    assert O.rho1(z) == pytest.approx((O.rho(z + h) - O.rho(z - h)) / (2 * h), rel=1e-8, abs=1e-9)
    assert O.rho2(z) == pytest.approx((O.rho1(z + h) - O.rho1(z - h)) / (2 * h), rel=1e-7, abs=1e-8)
    assert O.rho(z) == pytest.approx(math.log(1 + z * z), rel=1e-15)


# ----------------------------------------------------------------- padding and K (Eq. FOEmodel)

@pytest.mark.parametrize("n", [7, 8, 13])
def test_pad_index_matches_numpy_symmetric(n):
    ref = np.pad(np.arange(n), 3, mode="symmetric")
    got = [O.pad_index(i, n, O.BC_SYMMETRIC) for i in range(-3, n + 3)]
    assert got == list(ref)
    z = [O.pad_index(i, n, O.BC_ZERO) for i in range(-3, n + 3)]
    assert z == [-1] * 3 + list(range(n)) + [-1] * 3


@pytest.mark.parametrize("shape", [(8, 8), (13, 17), (40, 9)])
@pytest.mark.parametrize("bc", [O.BC_SYMMETRIC, O.BC_ZERO])
def test_responses_equal_library_convolution(bank, shape, bc):
    # Reading of Sec. 2.3: true convolution, responses at the N image pixels on a padded image.
    # scipy's 2-D convolution with 'symm' (edge repeated) or zero fill is the same operator.
    k, _ = bank
    rng = np.random.default_rng(1)
    u = rng.uniform(0, 5, shape)
    r = O.responses(k[:6], u, bc)
    for i in range(6):
        ref = signal.convolve2d(u, k[i], mode="same", boundary="symm" if bc == O.BC_SYMMETRIC else "fill")
        np.testing.assert_allclose(r[i], ref, rtol=0, atol=1e-12)
    # and the padded-valid form: np.pad + 'valid' convolution
    padded = np.pad(u, 3, mode="symmetric" if bc == O.BC_SYMMETRIC else "constant")
    np.testing.assert_allclose(r[0], signal.convolve2d(padded, k[0], mode="valid"), atol=1e-12)


@pytest.mark.parametrize("shape", [(8, 8), (13, 17), (7, 30)])
@pytest.mark.parametrize("bc", [O.BC_SYMMETRIC, O.BC_ZERO])
def test_adjoint_identity(bank, shape, bc):
    # <K u, psi> = <u, K^T psi> for the stacked operator K = (K_1; ...; K_nf), to FP64 rounding.
    k, _ = bank
    rng = np.random.default_rng(2)
    u = rng.standard_normal(shape)
    psi = rng.standard_normal((48,) + shape)
    lhs = float((O.responses(k, u, bc) * psi).sum())
    rhs = float((u * O.adjoint(k, psi, bc)).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-10)


@pytest.mark.parametrize("bc", [O.BC_SYMMETRIC, O.BC_ZERO])
def test_adjoint_is_dense_transpose_on_8x8(bank, bc):
    # Brute force: build each K_i as a dense 64x64 matrix from scipy's convolution of unit images
    # (independent of the oracle), then K_i^T psi must equal the oracle's adjoint.
    k, _ = bank
    H = W = 8
    rng = np.random.default_rng(3)
    psi = rng.standard_normal((3, H, W))
    expect = np.zeros(H * W)
    for i in range(3):
        M = np.zeros((H * W, H * W))
        for j in range(H * W):
            e = np.zeros(H * W)
            e[j] = 1.0
            M[:, j] = signal.convolve2d(e.reshape(H, W), k[i], mode="same",
                                        boundary="symm" if bc == O.BC_SYMMETRIC else "fill").ravel()
        expect += M.T @ psi[i].ravel()
    np.testing.assert_allclose(O.adjoint(k[:3], psi, bc).ravel(), expect, atol=1e-12)


def test_constant_image_has_zero_responses_under_symmetric_padding(bank):
    k, a = bank
    u = np.full((11, 14), 3.7)
    assert np.abs(O.responses(k, u, O.BC_SYMMETRIC)).max() < 1e-13
    assert np.abs(O.prior_grad(k, a, u, O.BC_SYMMETRIC)).max() < 1e-12


# ----------------------------------------------------------------- prior gradient (Eq. FoEF)

@pytest.mark.parametrize("bc", [O.BC_SYMMETRIC, O.BC_ZERO])
def test_prior_gradient_matches_finite_differences_8x8(bank, bc):
    k, a = bank
    rng = np.random.default_rng(4)
    u = rng.uniform(0, 4, (8, 8))
    g = O.prior_grad(k, a, u, bc)
    h = 1e-5
    fd = np.zeros_like(u)
    for idx in np.ndindex(u.shape):
        up, um = u.copy(), u.copy()
        up[idx] += h
        um[idx] -= h
        fd[idx] = (O.prior_energy(k, a, up, bc) - O.prior_energy(k, a, um, bc)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6)


def test_prior_gradient_matches_finite_differences_64x64_sampled(bank):
    k, a = bank
    rng = np.random.default_rng(5)
    u = rng.uniform(0, 6, (64, 64))
    g = O.prior_grad(k, a, u)
    h = 1e-5
    for _ in range(12):
        idx = (int(rng.integers(64)), int(rng.integers(64)))
        up, um = u.copy(), u.copy()
        up[idx] += h
        um[idx] -= h
        fd = (O.prior_energy(k, a, up) - O.prior_energy(k, a, um)) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-5)


def test_prior_gradient_small_signal_closed_form(bank):
    # For equal weights a and the orthonormal zero-mean bank (sum_i k_i k_i^T = I - 11^T/49 in tap
    # space), rho'(z) ~ 2z gives, away from the border,
    #   grad F(eps u) / eps -> 2a (49 u - B^T B u / 49),  B = 7x7 box sum.
    k, _ = bank
    a = 0.8
    rng = np.random.default_rng(6)
    u = rng.standard_normal((30, 30))
    eps = 1e-5
    g = O.prior_grad(k, np.full(48, a), eps * u, O.BC_ZERO) / eps
    box = np.ones((7, 7))
    Bu = signal.convolve2d(u, box, mode="same")
    BtBu = signal.convolve2d(Bu, box, mode="same")
    ref = 2 * a * (49 * u - BtBu / 49)
    np.testing.assert_allclose(g[6:-6, 6:-6], ref[6:-6, 6:-6], rtol=1e-6, atol=1e-6)


# ----------------------------------------------------------------- data terms and prox

@pytest.mark.parametrize("model", [O.MODEL_DIRECT, O.MODEL_ANS_L2, O.MODEL_ANS_IDIV])
def test_data_gradient_matches_finite_differences(model):
    rng = np.random.default_rng(7)
    u = rng.uniform(0.5, 5, 10)
    d = rng.integers(0, 6, 10).astype(float)
    g = O.data_grad(model, 1.7, u, d)
    h = 1e-6
    for i in range(10):
        up, um = u.copy(), u.copy()
        up[i] += h
        um[i] -= h
        fd = (O.data_energy(model, 1.7, up, d) - O.data_energy(model, 1.7, um, d)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-7)


@pytest.mark.parametrize("model", [O.MODEL_DIRECT, O.MODEL_ANS_L2])
def test_prox_is_the_argmin(model):
    # Eq. subproblemG: prox(ut) = argmin_u |u - ut|^2 / 2 + tau G(u), found by bounded 1-D search.
    rng = np.random.default_rng(8)
    tl = 0.37
    for _ in range(20):
        ut = float(rng.uniform(-2, 8))
        d = float(rng.integers(0, 9)) if model == O.MODEL_DIRECT else float(rng.uniform(1.2, 6))
        if model == O.MODEL_DIRECT:
            def obj(u):
                if u <= 0:
                    return 0.5 * (u - ut) ** 2 + (tl * u if d == 0 else np.inf)
                return 0.5 * (u - ut) ** 2 + tl * (u - d * math.log(u))
            lo = 0.0
        else:
            def obj(u):
                return 0.5 * (u - ut) ** 2 + tl * 0.5 * (u - d) ** 2
            lo = -10.0
        res = optimize.minimize_scalar(obj, bounds=(lo, 20.0), method="bounded",
                                       options={"xatol": 1e-11, "maxiter": 2000})
        got = O.prox(model, tl, np.array([ut]), np.array([d]))[0]
        assert got == pytest.approx(res.x, abs=2e-6)


def test_prox_fixed_point_at_data():
    # With ut = d the data-term prox returns d (both forms): the reason u^0 = d is a fixed point of
    # the data part alone.
    d = np.array([0.0, 1.0, 3.0, 17.0])
    assert np.allclose(O.prox(O.MODEL_DIRECT, 0.2, d, d), d, atol=1e-14)
    assert np.allclose(O.prox(O.MODEL_ANS_L2, 0.2, d, d), d, atol=1e-14)


# ----------------------------------------------------------------- step size

def test_lipschitz_closed_form_for_equal_weights(bank):
    # sum_i |k_i^(w)|^2 = 49 - |box^(w)|^2 / 49 for the orthonormal zero-mean bank, so
    # max_w = 49 (reached where the box symbol vanishes) and L = 2 kappa 49 a.
    k, _ = bank
    a = 1.3
    for bc, kappa in ((O.BC_SYMMETRIC, 4.0), (O.BC_ZERO, 1.0)):
        L = O.lipschitz(k, np.full(48, a), bc, ngrid=490)  # the grid contains 2 pi j / 7
        assert L == pytest.approx(2 * kappa * 49 * a, rel=1e-12)


def test_lipschitz_bounds_power_iteration(bank):
    # 2 ||sum_i alpha_i K_i^T K_i|| (power iteration on the oracle's own K, K^T) <= L.
    k, a = bank
    rng = np.random.default_rng(9)
    for bc in (O.BC_SYMMETRIC, O.BC_ZERO):
        u = rng.standard_normal((24, 24))
        lam = 0.0
        for _ in range(60):
            v = O.adjoint(k, O.responses(k, u, bc) * a[:, None, None], bc)
            lam = float(np.linalg.norm(v))
            u = v / lam
        assert 2 * lam <= O.lipschitz(k, a, bc, 256) * (1 + 1e-6)


# ----------------------------------------------------------------- iPiano (Eq. iPianoupdate)

def _tau(k, a, bc, gamma):
    return 0.99 * 2 * (1 - gamma) / (O.lipschitz(k, a, bc, 256) + 2e-3)


@pytest.mark.parametrize("model", [O.MODEL_DIRECT, O.MODEL_ANS_L2, O.MODEL_ANS_IDIV])
@pytest.mark.parametrize("bc", [O.BC_SYMMETRIC, O.BC_ZERO])
def test_ipiano_lyapunov_decrease(bank, model, bc):
    # With tau <= 2 (1 - gamma) / L, H(u^n, u^{n-1}) = E(u^n) + gamma / (2 tau) |u^n - u^{n-1}|^2
    # never increases (descent lemma + prox optimality).
    k, a = bank
    gamma = 0.8
    tau = _tau(k, a, bc, gamma)
    clean = synth.clean_image(24, 20, 11)
    y = synth.poisson_observation(clean, 4.0, 12)
    d = y if model == O.MODEL_DIRECT else O.anscombe(y)
    pr = O.Problem(k, a, 24, 20, bc=bc, model=model, lam=1.0, tau=tau, gamma=gamma)
    u, up = d.copy(), d.copy()
    Hs = []
    for _ in range(40):
        un = pr.step(d, u, up)
        up, u = u, un
        Hs.append(pr.energy(u, d) + gamma / (2 * tau) * float(((u - up) ** 2).sum()))
    Hs = np.array(Hs)
    assert np.all(np.diff(Hs) <= 1e-9 * np.abs(Hs[1:]))
    assert Hs[-1] < Hs[0]


def test_ipiano_without_inertia_decreases_energy(bank):
    k, a = bank
    tau = _tau(k, a, O.BC_SYMMETRIC, 0.0)
    y = synth.poisson_observation(synth.clean_image(16, 16, 13), 8.0, 14)
    d = O.anscombe(y)
    pr = O.Problem(k, a, 16, 16, model=O.MODEL_ANS_L2, lam=1.0, tau=tau, gamma=0.0)
    _, _, e = pr.ipiano(d, d, d, 30, trace=True)
    assert np.all(np.diff(e) <= 1e-12 * np.abs(e[1:]))


def test_ipiano_converges_to_stationary_point_8x8(bank):
    # At convergence u = prox(u - tau grad F(u)) (first-order optimality of F + G).
    k, a = bank
    gamma = 0.8
    tau = _tau(k, a, O.BC_SYMMETRIC, gamma)
    y = synth.poisson_observation(synth.clean_image(8, 8, 15), 4.0, 16)
    d = O.anscombe(y)
    pr = O.Problem(k, a, 8, 8, model=O.MODEL_ANS_L2, lam=1.0, tau=tau, gamma=gamma, nthreads=1)
    u, _ = pr.ipiano(d, d, d, 20000)
    res = O.prox(O.MODEL_ANS_L2, tau, u - tau * O.prior_grad(k, a, u, nthreads=1), d) - u
    assert np.abs(res).max() < 1e-9
    # the limit is also a zero of the full gradient
    _, g = pr.energy_grad(u, d)
    assert np.abs(g).max() < 1e-5


@pytest.mark.parametrize("model", [O.MODEL_ANS_L2, O.MODEL_ANS_IDIV])
def test_ipiano_stationary_point_at_lambda_not_one(bank, model):
    # lambda = 2.5: the limit solves grad R(u) + lambda grad D(u) = 0 with grad D written from the data terms of
    # Eq. subproblemGL2 (u - d) and Eq. subproblemGIdiv (1 - d / u), and it is a local minimum of E = R + lambda D.
    # A lambda dropped from the step's prox, from data_grad or from data_energy fails one of the three checks.
    k, a = bank
    lam, gamma = 2.5, 0.8
    tau = _tau(k, a, O.BC_SYMMETRIC, gamma)
    y = synth.poisson_observation(synth.clean_image(8, 8, 15), 4.0, 16)
    d = O.anscombe(y)
    pr = O.Problem(k, a, 8, 8, model=model, lam=lam, tau=tau, gamma=gamma, nthreads=1)
    u, _ = pr.ipiano(d, d, d, 20000)
    gd = (u - d) if model == O.MODEL_ANS_L2 else (1.0 - d / u)
    gr = O.prior_grad(k, a, u, nthreads=1)
    assert np.abs(gr + lam * gd).max() < 1e-6 * (1 + np.abs(gr).max())
    assert np.abs(gr + gd).max() > 1e-2            # the lambda = 1 condition does not hold there
    _, g = pr.energy_grad(u, d)
    assert np.abs(g).max() < 1e-5
    e0 = pr.energy(u, d)
    rng = np.random.default_rng(5)
    for _ in range(8):
        v = rng.standard_normal(u.shape)
        assert pr.energy(u + 1e-3 * v, d) > e0
    # the energy's data part scales with lambda: E_lam(u) - E_1(u) = (lam - 1) D(u), D taken at lambda = 1
    pr1 = O.Problem(k, a, 8, 8, model=model, lam=1.0, tau=tau, gamma=gamma, nthreads=1)
    dat = 0.5 * float(((u - d) ** 2).sum()) if model == O.MODEL_ANS_L2 else float((u - d * np.log(u)).sum())
    assert e0 - pr1.energy(u, d) == pytest.approx((lam - 1) * dat, rel=1e-10)


# ----------------------------------------------------------------- stopping rule (reading of Sec. 5.1)


def _data_only_stop(e0, gamma, tl, dn2, dv, vn2, tol, every, iters):
    # With no prior (alpha = 0) and the quadratic data term, u^0 = u^{-1} = d + e0 v stays on the line d + e v:
    # the prox of Eq. subproblemGL2 maps the inertial point d + (e_n + gamma (e_n - e_{n-1})) v to
    # d + (e_n + gamma (e_n - e_{n-1})) / (1 + tau lambda) v.  Then |u^n - u^{n-1}| = |e_n - e_{n-1}| |v| and
    # |u^n|^2 = |d|^2 + 2 e_n <d, v> + e_n^2 |v|^2, so the stopping step follows from the scalar recurrence.
    e_prev, e = e0, e0
    for n in range(1, iters + 1):
        e_prev, e = e, (e + gamma * (e - e_prev)) / (1 + tl)
        if n % every == 0 and abs(e - e_prev) * math.sqrt(vn2) <= tol * math.sqrt(dn2 + 2 * e * dv + e * e * vn2):
            return n, e
    return iters, e


@pytest.mark.parametrize("tol,every", [(1e-3, 5), (3e-5, 1), (1e-6, 7), (0.2, 3)])
def test_stopping_rule_data_only_closed_form(bank, tol, every):
    k, a = bank
    H = W = 10
    lam, tau, gamma = 3.0, 0.05, 0.8
    rng = np.random.default_rng(21)
    d = rng.uniform(1.0, 6.0, (H, W))
    v = rng.standard_normal((H, W))
    pr = O.Problem(k, np.zeros_like(a), H, W, model=O.MODEL_ANS_L2, lam=lam, tau=tau, gamma=gamma, nthreads=1)
    u0 = d + 1.0 * v
    u, up, n = pr.ipiano_tol(d, u0, u0, 400, tol, every)
    n_ref, e_ref = _data_only_stop(1.0, gamma, tau * lam, float((d * d).sum()), float((d * v).sum()),
                                   float((v * v).sum()), tol, every, 400)
    assert n == n_ref and 0 < n < 400 and n % every == 0
    np.testing.assert_allclose(u, d + e_ref * v, rtol=0, atol=1e-12)


def test_stopping_rule_special_cases(bank):
    k, a = bank
    y = synth.poisson_observation(synth.clean_image(12, 12, 31), 4.0, 32)
    d = O.anscombe(y)
    pr = O.Problem(k, a, 12, 12, model=O.MODEL_ANS_L2, lam=1.0, tau=1e-3, gamma=0.8, nthreads=1)
    u_full, up_full = pr.ipiano(d, d, d, 30)
    # tol = 0 never stops early, and a check interval beyond iters never checks: both equal the fixed-budget solve
    for tol, every in [(0.0, 1), (10.0, 31)]:
        u, up, n = pr.ipiano_tol(d, d, d, 30, tol, every)
        assert n == 30 and np.array_equal(u, u_full) and np.array_equal(up, up_full)
    # |u^n - u^{n-1}| <= |u^n| + |u^{n-1}|, so a tolerance above 1 + |u^{n-1}| / |u^n| stops at the first check
    u, _, n = pr.ipiano_tol(d, d, d, 30, 10.0, 4)
    u4, _ = pr.ipiano(d, d, d, 4)
    assert n == 4 and np.array_equal(u, u4)
    # the whole denoiser with the rule equals the fixed-budget denoiser run for the steps it took
    x, used, n = pr.denoise_tol(y, 4.0, 300, 2e-4, 10)
    assert 0 < n < 300 and n % 10 == 0
    xr, _ = pr.denoise(y, 4.0, n)
    assert np.array_equal(x, xr)


def test_denoise_model_selection_and_pipeline(bank):
    # Eq. FOEscheme: peak >= 5 -> quadratic data term, peak < 5 -> I-divergence (Anscombe domain).
    k, a = bank
    y = synth.poisson_observation(synth.clean_image(12, 12, 17), 4.0, 18)
    pr = O.Problem(k, a, 12, 12, model=O.MODEL_AUTO, lam=1.0, tau=1e-3, gamma=0.8, nthreads=1)
    assert pr.denoise(y, 4.99, 3)[1] == O.MODEL_ANS_IDIV
    assert pr.denoise(y, 5.0, 3)[1] == O.MODEL_ANS_L2
    # zero iterations: the output is the inverse transform of the data (Anscombe models) or the
    # zero-replaced data (direct model, Sec. 3.1.1)
    x, _ = pr.denoise(y, 5.0, 0)
    np.testing.assert_allclose(x, O.inverse(O.anscombe(y)), atol=1e-14)
    prd = O.Problem(k, a, 12, 12, model=O.MODEL_DIRECT, lam=1.0, tau=1e-3, gamma=0.8, nthreads=1)
    x, _ = prd.denoise(y, 4.0, 0, zero_c=0.1)
    np.testing.assert_allclose(x, np.where(y == 0, 0.1, y), atol=0)


def test_psnr_closed_form():
    a = np.full(100, 2.0)
    assert O.psnr(a + 0.1, a, 4.0) == pytest.approx(20 * math.log10(4.0 / 0.1), rel=1e-12)


# ----------------------------------------------------------------- training gradient (Sec. 2.5, 3.2)

@pytest.mark.parametrize("bc", [O.BC_SYMMETRIC, O.BC_ZERO])
def test_training_gradient_matches_central_differences(bank, bc):
    # Reverse-mode gradient of sum_s 1/2 ||I_C(u_s^T) - g_s||^2 through T unrolled steps against central
    # finite differences (eps = 1e-3, FP64) along random directions in (filters, log-weights).
    k, a = bank
    k, a = k[:6].copy(), a[:6].copy()
    H, W, T, B = 11, 9, 5, 2
    rng = np.random.default_rng(21)
    clean = np.stack([synth.clean_image(H, W, 30 + s) * 4.0 for s in range(B)])
    noisy = np.stack([synth.poisson_observation(clean[s] / 4.0, 4.0, 40 + s) for s in range(B)])
    tau = 0.02
    pr = O.Problem(k, a, H, W, bc=bc, model=O.MODEL_ANS_L2, lam=1.3, tau=tau, gamma=0.7, nthreads=1)
    L, dk, da = pr.train_grad(clean, noisy, T)
    assert L == pytest.approx(pr.train_loss(clean, noisy, T), rel=1e-14)
    eps = 1e-3
    for _ in range(3):
        dkd = rng.standard_normal(k.shape)
        dad = rng.standard_normal(a.shape)
        nrm = np.sqrt((dkd ** 2).sum() + (dad ** 2).sum())  # unit direction: the step is eps in parameter norm
        dkd, dad = dkd / nrm, dad / nrm
        def loss_at(t):
            q = O.Problem(k + t * dkd, a * np.exp(t * dad), H, W, bc=bc, model=O.MODEL_ANS_L2, lam=1.3, tau=tau,
                          gamma=0.7, nthreads=1)
            return q.train_loss(clean, noisy, T)
        fd = (loss_at(eps) - loss_at(-eps)) / (2 * eps)
        fd2 = (loss_at(eps / 2) - loss_at(-eps / 2)) / eps
        rich = (4 * fd2 - fd) / 3  # Richardson: removes the O(eps^2) truncation error of the central difference
        an = float((dk * dkd).sum() + (da * dad).sum())
        assert an == pytest.approx(fd, rel=1e-4, abs=1e-9)
        assert an == pytest.approx(rich, rel=1e-6, abs=1e-10)


# ------------------------------------------------- step control: Lipschitz backtracking (step a9)

def test_descent_lemma_at_the_certified_bound(bank):
    # L^ bounds the Lipschitz constant of grad F, so F(v) <= F(u) + <grad F(u), v - u> + L^/2 |v - u|^2 for every
    # u, v.  Along -g and +g the first-order term is the oracle's own gradient: a scaled or wrong gradient
    # violates the inequality for small steps, a wrong L^ (too small) for large ones.
    k, a = bank
    rng = np.random.default_rng(5)
    for bc in (O.BC_SYMMETRIC, O.BC_ZERO):
        Lh = O.lipschitz(k, a, bc, 256)
        for trial in range(3):
            u = rng.uniform(0.5, 8.0, (20, 18))
            F = O.prior_energy(k, a, u, bc)
            g = O.prior_grad(k, a, u, bc)
            for h in (-g, g, rng.standard_normal(u.shape)):
                for eps in (1e-4, 1e-2, 1.0 / Lh, 3.0 / Lh):
                    v = u + eps * h
                    rhs = F + float(np.sum(g * (v - u))) + 0.5 * Lh * float(np.sum((v - u) ** 2))
                    assert O.prior_energy(k, a, v, bc) <= rhs + 1e-10 * abs(F)


def test_backtracking_never_rejects_above_the_bound(bank):
    # Started high enough that L stays >= L^ for every step (it only shrinks by 1.5 per accepted step), the
    # descent lemma makes every trial acceptable: no L is ever doubled.
    k, a = bank
    H, W, iters = 20, 18, 12
    y = synth.poisson_observation(synth.clean_image(H, W, 21), 4.0, 22)
    d = O.anscombe(y)
    Lh = O.lipschitz(k, a, O.BC_SYMMETRIC, 256)
    pr = O.Problem(k, a, H, W, model=O.MODEL_ANS_L2, lam=1.0, gamma=0.8)
    _, _, trials = pr.ipiano_backtrack(d, d, iters, Lh * 1.5 ** iters)
    assert len(trials) == iters and all(ok for _, ok, _ in trials)


def test_backtracking_from_a_small_estimate(bank):
    # From an L far below the curvature the first trials are rejected and L doubles until the test passes;
    # each accepted step satisfies the sufficient-decrease inequality, the energy E = F + G decreases overall,
    # and replaying the accepted step sizes with fixed-step iPiano reproduces the iterates exactly.
    k, a = bank
    H, W, iters = 20, 18, 15
    y = synth.poisson_observation(synth.clean_image(H, W, 23), 4.0, 24)
    d = O.anscombe(y)
    Lh = O.lipschitz(k, a, O.BC_SYMMETRIC, 256)
    pr = O.Problem(k, a, H, W, model=O.MODEL_ANS_L2, lam=1.0, gamma=0.8)
    u, _, trials = pr.ipiano_backtrack(d, d, iters, Lh / 300.0)
    assert sum(1 for _, ok, _ in trials if not ok) >= 5
    assert sum(1 for _, ok, _ in trials if ok) == iters
    assert pr.energy(u, d) < pr.energy(d, d)
    taus = [t for t, ok, _ in trials if ok]
    v, vp = d.copy(), d.copy()
    for t in taus:
        vn = pr.step(d, v, vp, tau=t)
        vp, v = v, vn
    assert np.array_equal(v, u)
    # the recorded trials obey the rule: a rejection doubles L, an acceptance divides it by 1.5
    for (t0, ok0, L0), (t1, ok1, L1) in zip(trials, trials[1:]):
        assert math.isclose(L1, L0 * 2.0 if not ok0 else L0 / 1.5, rel_tol=1e-12)
        assert math.isclose(t0, 2 * (1 - 0.8) / (L0 + 2e-3), rel_tol=1e-12)


# ---- binning variant (FoEPNRbin, Sec. 4: 3x3 ones-kernel bins, bilinear upscaling) ----
@pytest.mark.parametrize("shape", [(9, 12), (8, 10), (7, 11)])
def test_bin3_one_hot_positions_and_border_scaling(shape):
    # a unit count at (r, c) lands in bin (r // 3, c // 3) alone, as 9 / n for a bin of n pixels (n < 9 only
    # where the border cuts the bin): pins the bin grid, the sum and the border reading
    H, W = shape
    Hb, Wb = (H + 2) // 3, (W + 2) // 3
    for r in range(H):
        for c in range(W):
            y = np.zeros((H, W))
            y[r, c] = 1.0
            yb = O.bin3(y)
            assert yb.shape == (Hb, Wb)
            I, J = r // 3, c // 3
            n = min(3, H - 3 * I) * min(3, W - 3 * J)
            want = np.zeros((Hb, Wb))
            want[I, J] = 9.0 / n
            np.testing.assert_array_equal(yb, want)


def test_bin3_raises_the_peak_nine_fold():
    # a constant image of c counts bins to 9c everywhere (border bins included); on a 3-divisible image the counts
    # are preserved in total
    np.testing.assert_array_equal(O.bin3(np.full((10, 14), 2.0)), np.full((4, 5), 18.0))
    y = np.random.default_rng(3).poisson(1.5, (12, 15)).astype(float)
    assert O.bin3(y).sum() == y.sum()


def test_upscale3_equals_library_bilinear_interpolation():
    # bilinear interpolation of the bin image at ((r - 1) / 3, (c - 1) / 3), clamped at the edges, is the order-1
    # spline of scipy.ndimage.map_coordinates with mode "nearest"
    from scipy import ndimage
    rng = np.random.default_rng(5)
    for H, W in [(21, 23), (19, 27), (30, 30)]:
        xb = rng.uniform(0.0, 9.0, ((H + 2) // 3, (W + 2) // 3))
        rr, cc = np.meshgrid((np.arange(H) - 1) / 3.0, (np.arange(W) - 1) / 3.0, indexing="ij")
        want = ndimage.map_coordinates(xb, [rr, cc], order=1, mode="nearest") / 9.0
        np.testing.assert_allclose(O.upscale3(xb, H, W), want, rtol=0, atol=1e-13)


def test_upscale3_reproduces_affine_images_between_bin_centres():
    # bin values sampled from an affine function at the bin centres (3I + 1, 3J + 1) come back as that function
    # (divided by 9) at every pixel whose interpolation stencil lies between centres
    H, W = 22, 25
    Hb, Wb = (H + 2) // 3, (W + 2) // 3
    f = lambda r, c: 9.0 * (0.7 + 0.11 * r - 0.05 * c)
    I, J = np.meshgrid(np.arange(Hb), np.arange(Wb), indexing="ij")
    x = O.upscale3(f(3 * I + 1.0, 3 * J + 1.0), H, W)
    r, c = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    inside = (r >= 1) & (r <= 3 * (Hb - 1) + 1) & (c >= 1) & (c <= 3 * (Wb - 1) + 1)
    np.testing.assert_allclose(x[inside], f(r, c)[inside] / 9.0, rtol=0, atol=1e-13)


def test_denoise_binned_constant_image_and_binned_peak_threshold(bank):
    # a constant image of c counts bins to the constant 9c, a stationary point of the prior (zero-mean filters) and
    # of the quadratic data term at u = v: the result is I_C(2 sqrt(9c + 3/8)) / 9 everywhere.  The data term is
    # chosen by the binned peak, 9 * peak, against the threshold 5 (Sec. 3.4).
    k, a = bank
    H, W = 20, 23
    pr = O.Problem(k, a, H, W, model=O.MODEL_AUTO, lam=1.0, tau=1e-3, gamma=0.8, nthreads=1)
    x, used = pr.denoise_binned(np.full((H, W), 3.0), 0.6, 20)
    assert used == O.MODEL_ANS_L2
    want = float(O.inverse(np.array([2.0 * math.sqrt(27.0 + 3.0 / 8.0)]))[0]) / 9.0
    np.testing.assert_allclose(x, want, rtol=1e-12)
    y = synth.poisson_observation(synth.clean_image(H, W, 19), 0.5, 20)
    assert pr.denoise_binned(y, 0.5, 2)[1] == O.MODEL_ANS_IDIV
    assert pr.denoise_binned(y, 5.0 / 9.0, 2)[1] == O.MODEL_ANS_L2


# ------------------------------------- the paper's training gradient by implicit differentiation (Sec. 2.5)

def _small_training_problem(bank, H=8, W=9, nf=6, lam=1.0, gamma=0.8, bc=O.BC_SYMMETRIC):
    k, a = bank
    k, a = k[:nf].copy(), a[:nf].copy()
    tau = 0.99 * 2 * (1 - gamma) / (O.lipschitz(k, a, bc) + 2e-3)
    return k, a, tau, O.Problem(k, a, H, W, bc=bc, model=O.MODEL_ANS_L2, lam=lam, tau=tau, gamma=gamma, nthreads=1)


@pytest.mark.parametrize("bc", [O.BC_SYMMETRIC, O.BC_ZERO])
def test_hessian_vector_product_matches_gradient_differences(bank, bc):
    # H_E(w) x = d/dt grad E(w + t x) at t = 0 (central differences of the oracle's gradient, FP64)
    k, a, tau, pr = _small_training_problem(bank, H=10, W=9, bc=bc)
    rng = np.random.default_rng(8)
    d = O.anscombe(rng.poisson(3.0, (10, 9)).astype(float))
    w = d + rng.normal(0.0, 0.3, d.shape)
    x = rng.standard_normal(d.shape)
    eps = 1e-5
    fd = (pr.energy_grad(w + eps * x, d)[1] - pr.energy_grad(w - eps * x, d)[1]) / (2 * eps)
    hv = pr.hvp(w, x)
    assert np.abs(hv - fd).max() <= 1e-6 * np.abs(hv).max()


def test_conjugate_gradients_match_a_dense_solve(bank):
    # H_E assembled column by column from the product and solved by LAPACK; CG from 0 reaches the same q
    k, a, tau, pr = _small_training_problem(bank, H=8, W=9)
    rng = np.random.default_rng(9)
    w = O.anscombe(rng.poisson(3.0, (8, 9)).astype(float))
    n = w.size
    Hd = np.stack([pr.hvp(w, np.eye(n)[j].reshape(w.shape)).ravel() for j in range(n)], axis=1)
    assert np.abs(Hd - Hd.T).max() <= 1e-12 * np.abs(Hd).max()
    b = rng.standard_normal(w.shape)
    q, it, rel = pr.cg(w, b, 500, 1e-13)
    assert rel <= 1e-13 and it <= 500
    np.testing.assert_allclose(q.ravel(), np.linalg.solve(Hd, b.ravel()), rtol=0, atol=1e-10 * np.abs(q).max())


def test_implicit_gradient_is_the_derivative_of_the_loss_at_the_minimiser(bank):
    # Eq. implicitdifferentiation / overallderivative at a tightly converged minimiser against (i) central
    # differences of the loss of the converged solve along random parameter directions and (ii) the unrolled
    # reverse-mode gradient of the same T steps, which tends to it as T grows
    k, a, tau, pr = _small_training_problem(bank)
    H, W, T, B = 8, 9, 3000, 2
    clean = np.stack([synth.clean_image(H, W, 50 + s) * 4.0 for s in range(B)])
    noisy = np.stack([synth.poisson_observation(clean[s] / 4.0, 4.0, 60 + s) for s in range(B)])
    L, dk, da, it, rel = pr.train_grad_implicit(clean, noisy, T, 400, 1e-13)
    assert rel <= 1e-12
    assert L == pytest.approx(pr.train_loss(clean, noisy, T), rel=1e-14)
    Lu, dku, dau = pr.train_grad(clean, noisy, T)
    g_imp = np.concatenate([dk.ravel(), da])
    g_unr = np.concatenate([dku.ravel(), dau])
    assert np.abs(g_imp - g_unr).max() <= 1e-7 * np.abs(g_imp).max()
    rng = np.random.default_rng(22)
    eps = 1e-4
    for _ in range(3):
        dkd = rng.standard_normal(k.shape)
        dad = rng.standard_normal(a.shape)
        nrm = np.sqrt((dkd ** 2).sum() + (dad ** 2).sum())
        dkd, dad = dkd / nrm, dad / nrm

        def loss_at(t):
            q = O.Problem(k + t * dkd, a * np.exp(t * dad), H, W, model=O.MODEL_ANS_L2, lam=1.0, tau=tau, gamma=0.8,
                          nthreads=1)
            return q.train_loss(clean, noisy, T)
        fd = (loss_at(eps) - loss_at(-eps)) / (2 * eps)
        an = float((dk * dkd).sum() + (da * dad).sum())
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-10)
