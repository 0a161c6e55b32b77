"""FP64 oracle of the FoE Poisson denoiser: ctypes wrapper around ``foe_oracle.c``.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline legs may import this package.  The CUDA library never loads it
and it never loads the CUDA library.

The C file is compiled here with gcc (``-O3 -ffp-contract=off``, no fast-math, so the FP64
results are the same on x86-64 and aarch64 hosts).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "foe_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None

MODEL_DIRECT, MODEL_ANS_L2, MODEL_ANS_IDIV, MODEL_AUTO = 0, 1, 2, 3
BC_SYMMETRIC, BC_ZERO = 0, 1

_dp = C.POINTER(C.c_double)


class Params(C.Structure):
    _fields_ = [
        ("nf", C.c_int), ("k", _dp), ("alpha", _dp),
        ("H", C.c_int), ("W", C.c_int), ("bc", C.c_int), ("model", C.c_int),
        ("lam", C.c_double), ("tau", C.c_double), ("gamma", C.c_double),
        ("nthreads", C.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liborc.so`` (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O3", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11",
                    "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm", "-lpthread"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> C.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            for name in ("orc_anscombe1", "orc_ic1", "orc_ic_deriv1", "orc_rho", "orc_rho1", "orc_rho2"):
                getattr(L, name).restype = C.c_double
                getattr(L, name).argtypes = [C.c_double]
            L.orc_pad_index.restype = C.c_long
            L.orc_pad_index.argtypes = [C.c_long, C.c_long, C.c_int]
            L.orc_anscombe.argtypes = [C.c_long, _dp, _dp]
            L.orc_inverse.argtypes = [C.c_long, _dp, _dp]
            L.orc_responses.argtypes = [C.c_int, _dp, C.c_int, C.c_int, _dp, C.c_int, _dp, C.c_int]
            L.orc_adjoint.argtypes = [C.c_int, _dp, C.c_int, C.c_int, _dp, C.c_int, _dp, C.c_int]
            L.orc_prior_energy.restype = C.c_double
            L.orc_prior_energy.argtypes = [C.c_int, _dp, _dp, C.c_int, C.c_int, _dp, C.c_int, C.c_int]
            L.orc_prior_grad.argtypes = [C.c_int, _dp, _dp, C.c_int, C.c_int, _dp, C.c_int, _dp, C.c_int]
            L.orc_data_energy.restype = C.c_double
            L.orc_data_energy.argtypes = [C.c_int, C.c_double, C.c_long, _dp, _dp]
            L.orc_data_grad.argtypes = [C.c_int, C.c_double, C.c_long, _dp, _dp, _dp]
            L.orc_prox.argtypes = [C.c_int, C.c_double, C.c_long, _dp, _dp, _dp]
            L.orc_energy.restype = C.c_double
            L.orc_energy.argtypes = [C.POINTER(Params), _dp, _dp]
            L.orc_energy_grad.restype = C.c_double
            L.orc_energy_grad.argtypes = [C.POINTER(Params), _dp, _dp, _dp]
            L.orc_ipiano_step.argtypes = [C.POINTER(Params), _dp, _dp, _dp, _dp]
            L.orc_ipiano.restype = C.c_int
            L.orc_ipiano.argtypes = [C.POINTER(Params), _dp, _dp, _dp, C.c_int, _dp]
            L.orc_denoise.restype = C.c_int
            L.orc_denoise.argtypes = [C.POINTER(Params), _dp, C.c_double, C.c_double, C.c_int, _dp]
            L.orc_ipiano_tol.restype = C.c_int
            L.orc_ipiano_tol.argtypes = [C.POINTER(Params), _dp, _dp, _dp, C.c_int, C.c_double, C.c_int]
            L.orc_denoise_tol.restype = C.c_int
            L.orc_denoise_tol.argtypes = [C.POINTER(Params), _dp, C.c_double, C.c_double, C.c_int, C.c_double,
                                          C.c_int, _dp, C.POINTER(C.c_int)]
            L.orc_bin3.argtypes = [C.c_int, C.c_int, _dp, _dp]
            L.orc_upscale3.argtypes = [C.c_int, C.c_int, _dp, C.c_int, C.c_int, _dp]
            L.orc_denoise_binned.restype = C.c_int
            L.orc_denoise_binned.argtypes = [C.POINTER(Params), _dp, C.c_double, C.c_double, C.c_int, _dp]
            L.orc_lipschitz.restype = C.c_double
            L.orc_lipschitz.argtypes = [C.c_int, _dp, _dp, C.c_int, C.c_int]
            L.orc_train_loss.restype = C.c_double
            L.orc_train_loss.argtypes = [C.POINTER(Params), C.c_int, _dp, _dp, C.c_int]
            L.orc_train_grad.restype = C.c_double
            L.orc_train_grad.argtypes = [C.POINTER(Params), C.c_int, _dp, _dp, C.c_int, _dp, _dp]
            L.orc_hvp.argtypes = [C.POINTER(Params), _dp, _dp, _dp]
            L.orc_cg.restype = C.c_int
            L.orc_cg.argtypes = [C.POINTER(Params), _dp, _dp, C.c_int, C.c_double, _dp, _dp]
            L.orc_train_grad_implicit.restype = C.c_double
            L.orc_train_grad_implicit.argtypes = [C.POINTER(Params), C.c_int, _dp, _dp, C.c_int, C.c_int, C.c_double,
                                                  _dp, _dp, C.POINTER(C.c_int), _dp]
            L.orc_psnr.restype = C.c_double
            L.orc_psnr.argtypes = [C.c_long, _dp, _dp, C.c_double]
            _lib = L
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# ---- scalar maps (Eq. Anscombetransform, Eq. invAns, I_C', Eq. STfunc) ----
def anscombe(y):
    y = _d(y)
    v = np.empty_like(y)
    lib().orc_anscombe(y.size, _p(y), _p(v))
    return v


def inverse(z):
    z = _d(z)
    x = np.empty_like(z)
    lib().orc_inverse(z.size, _p(z), _p(x))
    return x


def ic(z: float) -> float:
    return lib().orc_ic1(float(z))


def ic_deriv(z: float) -> float:
    return lib().orc_ic_deriv1(float(z))


def rho(z: float) -> float:
    return lib().orc_rho(float(z))


def rho1(z: float) -> float:
    return lib().orc_rho1(float(z))


def rho2(z: float) -> float:
    return lib().orc_rho2(float(z))


def pad_index(i: int, n: int, bc: int) -> int:
    return lib().orc_pad_index(i, n, bc)


# ---- linear operators (Eq. FOEmodel, Sec. 2.5.2) ----
def _filters(k) -> np.ndarray:
    k = _d(k)
    return k.reshape(k.shape[0], 49)


def responses(k, u, bc=BC_SYMMETRIC, nthreads=None):
    k = _filters(k)
    u = _d(u)
    H, W = u.shape
    r = np.empty((k.shape[0], H, W))
    lib().orc_responses(k.shape[0], _p(k), H, W, _p(u), bc, _p(r), nthreads or default_threads())
    return r


def adjoint(k, psi, bc=BC_SYMMETRIC, nthreads=None):
    k = _filters(k)
    psi = _d(psi)
    nf, H, W = psi.shape
    g = np.empty((H, W))
    lib().orc_adjoint(nf, _p(k), H, W, _p(psi), bc, _p(g), nthreads or default_threads())
    return g


def prior_energy(k, alpha, u, bc=BC_SYMMETRIC, nthreads=None) -> float:
    k, a, u = _filters(k), _d(alpha), _d(u)
    H, W = u.shape
    return lib().orc_prior_energy(k.shape[0], _p(k), _p(a), H, W, _p(u), bc, nthreads or default_threads())


def prior_grad(k, alpha, u, bc=BC_SYMMETRIC, nthreads=None):
    k, a, u = _filters(k), _d(alpha), _d(u)
    H, W = u.shape
    g = np.empty((H, W))
    lib().orc_prior_grad(k.shape[0], _p(k), _p(a), H, W, _p(u), bc, _p(g), nthreads or default_threads())
    return g


def data_energy(model, lam, u, d) -> float:
    u, d = _d(u), _d(d)
    return lib().orc_data_energy(model, float(lam), u.size, _p(u), _p(d))


def data_grad(model, lam, u, d):
    u, d = _d(u), _d(d)
    g = np.empty_like(u)
    lib().orc_data_grad(model, float(lam), u.size, _p(u), _p(d), _p(g))
    return g


def prox(model, tl, ut, d):
    ut, d = _d(ut), _d(d)
    out = np.empty_like(ut)
    lib().orc_prox(model, float(tl), ut.size, _p(ut), _p(d), _p(out))
    return out


# ---- solver ----
class Problem:
    """Holds the parameter block and keeps its arrays alive."""

    def __init__(self, k, alpha, H, W, *, bc=BC_SYMMETRIC, model=MODEL_ANS_L2, lam=1.0, tau=1e-3,
                 gamma=0.8, nthreads=None):
        self.k = _filters(k)
        self.alpha = _d(alpha)
        self.p = Params(self.k.shape[0], _p(self.k), _p(self.alpha), int(H), int(W), int(bc), int(model),
                        float(lam), float(tau), float(gamma), int(nthreads or default_threads()))

    def energy(self, u, d) -> float:
        u, d = _d(u), _d(d)
        return lib().orc_energy(C.byref(self.p), _p(u), _p(d))

    def energy_grad(self, u, d):
        u, d = _d(u), _d(d)
        g = np.empty_like(u)
        e = lib().orc_energy_grad(C.byref(self.p), _p(u), _p(d), _p(g))
        return e, g

    def step(self, d, u, u_prev, tau=None):
        """One iPiano step (Sec. 2.3, Eq. iPianoupdate); tau, if given, replaces the problem's step size for
        this step only (the replay of a step-size sequence)."""
        d, u, up = _d(d), _d(u), _d(u_prev)
        un = np.empty_like(u)
        p = self.p
        if tau is not None:
            p = Params()
            C.memmove(C.byref(p), C.byref(self.p), C.sizeof(Params))
            p.tau = float(tau)
        lib().orc_ipiano_step(C.byref(p), _p(d), _p(u), _p(up), _p(un))
        return un

    def ipiano_backtrack(self, d, u0, iters, L0, c2=1e-3):
        """iPiano with Lipschitz backtracking on the smooth part F = E_FoE (Sec. 2.3 gives tau and gamma only as
        symbols; this is the backtracking rule of the iPiano method): a trial with estimate L takes
        tau = 2 (1 - gamma) / (L + 2 c2) and is accepted when
            F(u+) <= F(u) + <grad F(u), u+ - u> + L/2 ||u+ - u||^2,
        else L doubles and the trial is repeated from the same u; after an accepted step L is divided by 1.5.
        Returns (u, u_prev, trials) with trials a list of (tau, accepted, L)."""
        gamma = self.p.gamma
        k, a, bc = self.k, self.alpha, self.p.bc
        u = _d(u0).copy()
        up = u.copy()
        F = prior_energy(k, a, u, bc)
        L = float(L0)
        trials = []
        for _ in range(iters):
            g = prior_grad(k, a, u, bc)
            while True:
                tau = 2.0 * (1.0 - gamma) / (L + 2.0 * c2)
                un = self.step(d, u, up, tau=tau)
                du = un - u
                Fn = prior_energy(k, a, un, bc)
                ok = Fn <= F + float(np.sum(g * du)) + 0.5 * L * float(np.sum(du * du))
                trials.append((tau, ok, L))
                if ok:
                    break
                L *= 2.0
            up, u, F = u, un, Fn
            L /= 1.5
        return u, up, trials

    def ipiano(self, d, u0, u_prev0, iters, trace=False):
        d = _d(d)
        u = _d(u0).copy()
        up = _d(u_prev0).copy()
        e = np.empty(iters + 1) if trace else None
        lib().orc_ipiano(C.byref(self.p), _p(d), _p(u), _p(up), int(iters), _p(e) if trace else None)
        return (u, up, e) if trace else (u, up)

    def train_loss(self, clean, noisy, T) -> float:
        """Sum over the batch of 1/2 ||I_C(u^T) - g||^2 (Anscombe quadratic model, T unrolled steps)."""
        c, y = _d(clean), _d(noisy)
        return lib().orc_train_loss(C.byref(self.p), c.shape[0], _p(c), _p(y), int(T))

    def train_grad(self, clean, noisy, T):
        """(loss, dL/dk (nf, 7, 7) in convolution orientation, dL/d log alpha (nf,))."""
        c, y = _d(clean), _d(noisy)
        dk = np.empty((self.k.shape[0], 49))
        da = np.empty(self.k.shape[0])
        L = lib().orc_train_grad(C.byref(self.p), c.shape[0], _p(c), _p(y), int(T), _p(dk), _p(da))
        return L, dk.reshape(-1, 7, 7), da

    def hvp(self, w, x):
        """H_E(w) x for the Anscombe quadratic model: sum_i alpha_i K_i^T diag(rho''(K_i w)) K_i x + lambda x."""
        w, x = _d(w), _d(x)
        out = np.empty_like(w)
        lib().orc_hvp(C.byref(self.p), _p(w), _p(x), _p(out))
        return out

    def cg(self, w, b, max_cg, tol):
        """q ~ H_E(w)^{-1} b by conjugate gradients from 0: (q, iterations, relative residual)."""
        w, b = _d(w), _d(b)
        q = np.empty_like(w)
        rel = np.zeros(1)
        it = lib().orc_cg(C.byref(self.p), _p(w), _p(b), int(max_cg), float(tol), _p(q), _p(rel))
        return q, it, float(rel[0])

    def train_grad_implicit(self, clean, noisy, T, max_cg, tol):
        """(loss, dL/dk (nf, 7, 7), dL/d log alpha (nf,), max CG iterations, max relative residual) by Eq.
        implicitdifferentiation at u^T (T iPiano steps) for a batch of images (leading axis)."""
        c, y = _d(clean), _d(noisy)
        dk = np.empty((self.k.shape[0], 49))
        da = np.empty(self.k.shape[0])
        it = C.c_int(0)
        rel = np.zeros(1)
        L = lib().orc_train_grad_implicit(C.byref(self.p), c.shape[0], _p(c), _p(y), int(T), int(max_cg), float(tol),
                                          _p(dk), _p(da), C.byref(it), _p(rel))
        return L, dk.reshape(-1, 7, 7), da, it.value, float(rel[0])

    def denoise(self, y, peak, iters, zero_c=0.0):
        y = _d(y)
        x = np.empty_like(y)
        used = lib().orc_denoise(C.byref(self.p), _p(y), float(peak), float(zero_c), int(iters), _p(x))
        return x, used

    def ipiano_tol(self, d, u0, u_prev0, iters, tol, check_every):
        """At most iters steps, stopping after step n (a multiple of check_every) once ||u^n - u^{n-1}|| <=
        tol ||u^n||: (u, u_prev, steps taken)."""
        d = _d(d)
        u = _d(u0).copy()
        up = _d(u_prev0).copy()
        n = lib().orc_ipiano_tol(C.byref(self.p), _p(d), _p(u), _p(up), int(iters), float(tol), int(check_every))
        return u, up, n

    def denoise_tol(self, y, peak, iters, tol, check_every, zero_c=0.0):
        """denoise with the stopping rule of ipiano_tol: (x, model used, steps taken)."""
        y = _d(y)
        x = np.empty_like(y)
        done = C.c_int(0)
        used = lib().orc_denoise_tol(C.byref(self.p), _p(y), float(peak), float(zero_c), int(iters), float(tol),
                                     int(check_every), _p(x), C.byref(done))
        return x, used, done.value

    def denoise_binned(self, y, peak, iters, zero_c=0.0):
        """FoEPNRbin: bin3, denoise the binned image at 9 * peak, upscale3 (the problem's H, W are the full sizes)."""
        y = _d(y)
        x = np.empty_like(y)
        used = lib().orc_denoise_binned(C.byref(self.p), _p(y), float(peak), float(zero_c), int(iters), _p(x))
        return x, used


# ---- binning variant (FoEPNRbin, Sec. 4) ----
def bin3(y):
    """Sums of the non-overlapping 3x3 bins, ceil(H/3) x ceil(W/3); a bin cut by the border is scaled by 9 / n."""
    y = _d(y)
    H, W = y.shape
    yb = np.empty(((H + 2) // 3, (W + 2) // 3))
    lib().orc_bin3(H, W, _p(y), _p(yb))
    return yb


def upscale3(xb, H, W):
    """Bilinear interpolation of the bin image at ((r - 1) / 3, (c - 1) / 3), clamped to the edge bins, / 9."""
    xb = _d(xb)
    x = np.empty((int(H), int(W)))
    lib().orc_upscale3(xb.shape[0], xb.shape[1], _p(xb), int(H), int(W), _p(x))
    return x


def lipschitz(k, alpha, bc=BC_SYMMETRIC, ngrid=512) -> float:
    k, a = _filters(k), _d(alpha)
    return lib().orc_lipschitz(k.shape[0], _p(k), _p(a), bc, ngrid)


def psnr(a, b, peak) -> float:
    a, b = _d(a), _d(b)
    return lib().orc_psnr(a.size, _p(a), _p(b), float(peak))
