"""Thin Python binding of the C ABI in ``include/foe.h`` (ctypes; argument marshalling only).

Every function has the name of the C entry point it calls.  Device buffers are passed as
objects with ``data_ptr()`` (torch tensors) or as integer addresses; streams as a
``torch.cuda.Stream``, a raw handle or ``None`` (torch's current stream when torch is loaded,
else the legacy default stream).  All arithmetic runs in the CUDA library: if ``libfoe.so``
is missing, every call raises instead of computing anything on the host.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfoe.so")

FOE_OK, FOE_EINVAL, FOE_ENOMEM, FOE_ECUDA, FOE_ENONFINITE, FOE_ETIMEOUT, FOE_EBUSY, FOE_EUNSUPPORTED = range(8)
FOE_MODEL_DIRECT, FOE_MODEL_ANS_L2, FOE_MODEL_ANS_IDIV, FOE_MODEL_AUTO = range(4)
FOE_PREC_FP32, FOE_PREC_TF32, FOE_PREC_BF16 = range(3)
FOE_BC_SYMMETRIC, FOE_BC_ZERO = range(2)
FOE_STEP_FIXED, FOE_STEP_BACKTRACK = range(2)

_fp = C.POINTER(C.c_float)


class foe_prior(C.Structure):
    _fields_ = [("nf", C.c_int), ("ksize", C.c_int), ("filters", _fp), ("alpha", _fp)]


class foe_solve_opts(C.Structure):
    _fields_ = [("model", C.c_int), ("lam", C.c_float), ("gamma", C.c_float), ("tau", C.c_float),
                ("tol", C.c_float), ("iters", C.c_int), ("step", C.c_int), ("bc", C.c_int),
                ("prec", C.c_int), ("zero_c", C.c_float), ("use_graph", C.c_int), ("tol_every", C.c_int)]


class foe_report(C.Structure):
    _fields_ = [("iters_done", C.c_int), ("model_used", C.c_int), ("tau_used", C.c_float), ("status", C.c_int),
                ("backtracks", C.c_int), ("lipschitz_final", C.c_double), ("nonfinite", C.c_int)]


class foe_image_desc(C.Structure):
    _fields_ = [("y", C.c_void_p), ("x", C.c_void_p), ("H", C.c_int), ("W", C.c_int), ("ld", C.c_int),
                ("peak", C.c_float), ("iters", C.c_int), ("use_model", C.c_int), ("model", C.c_int)]


class foe_server_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_active", C.c_int), ("iters_per_tick", C.c_int),
                ("use_graphs", C.c_int), ("opts", foe_solve_opts)]


class foe_server_stats(C.Structure):
    _fields_ = [("queued", C.c_int), ("active", C.c_int), ("finishing", C.c_int), ("completed", C.c_longlong),
                ("ticks", C.c_longlong), ("launches", C.c_longlong), ("pixel_iters", C.c_double), ("bytes_in_use", C.c_size_t),
                ("bytes_peak", C.c_size_t), ("bytes_budget", C.c_size_t)]


class FoeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """Loads libfoe.so; raises if it has not been built (there is no host fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run paper_1609_05722_gb300.build)")
        L = C.CDLL(LIB_PATH)
        vp, i, f, d = C.c_void_p, C.c_int, C.c_float, C.c_double
        sig = {
            "foe_default_opts": (i, [C.POINTER(foe_solve_opts)]),
            "foe_create": (i, [C.POINTER(foe_prior), C.POINTER(vp)]),
            "foe_destroy": (None, [vp]),
            "foe_step_size": (i, [vp, i, f, C.POINTER(f), C.POINTER(d)]),
            "foe_prior_lipschitz": (i, [C.POINTER(foe_prior), i, C.POINTER(d)]),
            "foe_step_log": (i, [vp, C.POINTER(f), C.POINTER(C.c_ubyte), i]),
            "foe_denoise": (i, [vp, vp, vp, i, i, i, f, C.POINTER(foe_solve_opts), vp, C.POINTER(foe_report)]),
            "foe_device_status": (i, [vp, vp]),
            "foe_debug_withhold_arrival": (i, [vp]),
            "foe_denoise_binned": (i, [vp, vp, vp, i, i, i, f, C.POINTER(foe_solve_opts), vp, C.POINTER(foe_report)]),
            "foe_denoise_batch": (i, [vp, C.POINTER(foe_image_desc), i, C.POINTER(foe_solve_opts), vp]),
            "foe_iters_done": (i, [vp, C.POINTER(i), i, vp]),
            "foe_energy_grad": (i, [vp, vp, vp, i, i, i, i, f, i, i, C.POINTER(d), vp, vp]),
            "foe_ipiano_step": (i, [vp, vp, vp, vp, vp, vp, i, i, i, i, f, f, f, i, i, vp]),
            "foe_anscombe": (i, [vp, vp, C.c_long, vp]),
            "foe_inverse": (i, [vp, vp, C.c_long, vp]),
            "foe_denoise_static": (i, [vp, vp, vp, i, i, i, f, C.POINTER(foe_solve_opts), vp]),
            "foe_server_create": (i, [vp, C.POINTER(foe_server_config), C.POINTER(vp)]),
            "foe_server_destroy": (None, [vp]),
            "foe_server_submit": (i, [vp, vp, i, vp, i, i, i, f, i, C.POINTER(C.c_longlong)]),
            "foe_server_tick": (i, [vp, C.POINTER(i)]),
            "foe_server_poll": (i, [vp, C.POINTER(C.c_longlong), i, C.POINTER(i)]),
            "foe_server_get_stats": (i, [vp, C.POINTER(foe_server_stats)]),
            "foe_train_step": (i, [vp, vp, vp, i, i, i, i, C.POINTER(foe_solve_opts), i, C.POINTER(d), vp, vp, vp]),
            "foe_train_grad_implicit": (i, [vp, vp, vp, i, i, i, i, C.POINTER(foe_solve_opts), i, f, C.POINTER(d), vp,
                                            vp, C.POINTER(foe_implicit_report), vp]),
            "foe_profile": (i, [vp, i]),
            "foe_profile_read": (i, [vp, C.POINTER(d), C.POINTER(C.c_long), C.POINTER(d)]),
            "foe_mma_cost": (i, [i, i, i, i, i, i, C.POINTER(d)]),
            "foe_status_string": (C.c_char_p, [i]),
            "foe_last_error": (C.c_char_p, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> int | None:
    if s is None:
        import sys
        torch = sys.modules.get("torch")
        if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
            return int(torch.cuda.current_stream().cuda_stream)
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _check(status: int, ctx=None, what: str = ""):
    if status != FOE_OK:
        text = lib().foe_status_string(status).decode()
        if ctx is not None:
            text += ": " + lib().foe_last_error(ctx).decode()
        raise FoeError(status, f"{what}: {text}" if what else text)


def foe_status_string(status: int) -> str:
    return lib().foe_status_string(status).decode()


def foe_last_error(ctx) -> str:
    return lib().foe_last_error(ctx).decode()


def foe_device_status(ctx, stream=None) -> int:
    """Reads and clears the context's device-side status (FOE_OK or FOE_ETIMEOUT); synchronises the stream."""
    return lib().foe_device_status(ctx, _stream(stream))


def foe_debug_withhold_arrival(ctx) -> None:
    """Failure-detection test aid: the next tensor-core launch lets one bounded device wait expire."""
    _check(lib().foe_debug_withhold_arrival(ctx), ctx, "foe_debug_withhold_arrival")


@dataclass
class SolveOpts:
    """Python mirror of foe_solve_opts (defaults of foe_default_opts)."""
    model: int = FOE_MODEL_AUTO
    lam: float = 1.0
    gamma: float = 0.8
    tau: float = 0.0
    tol: float = 0.0
    iters: int = 300
    step: int = FOE_STEP_FIXED
    bc: int = FOE_BC_SYMMETRIC
    prec: int = FOE_PREC_BF16
    zero_c: float = 0.0
    use_graph: bool = False
    tol_every: int = 10

    def c(self) -> foe_solve_opts:
        return foe_solve_opts(self.model, self.lam, self.gamma, self.tau, self.tol, self.iters, self.step,
                              self.bc, self.prec, self.zero_c, 1 if self.use_graph else 0, self.tol_every)


def foe_default_opts() -> SolveOpts:
    o = foe_solve_opts()
    _check(lib().foe_default_opts(C.byref(o)))
    return SolveOpts(o.model, o.lam, o.gamma, o.tau, o.tol, o.iters, o.step, o.bc, o.prec, o.zero_c,
                     bool(o.use_graph), o.tol_every)


def _prior(filters, alpha):
    k = np.asarray(filters, dtype=np.float32)
    ks = k.shape[-1] if k.ndim == 3 else 7
    k = np.ascontiguousarray(k.reshape(k.shape[0], -1))
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float32).ravel())
    p = foe_prior(k.shape[0], ks, k.ctypes.data_as(_fp), a.ctypes.data_as(_fp))
    return p, (k, a)


def foe_prior_lipschitz(filters, alpha, bc: int = FOE_BC_SYMMETRIC) -> float:
    p, _keep = _prior(filters, alpha)
    out = C.c_double()
    _check(lib().foe_prior_lipschitz(C.byref(p), bc, C.byref(out)), what="foe_prior_lipschitz")
    return out.value


def foe_create(filters, alpha) -> int:
    """filters: (nf, 7, 7) convolution kernels k_i(a, b); alpha: (nf,) positive weights."""
    p, _keep = _prior(filters, alpha)
    h = C.c_void_p()
    _check(lib().foe_create(C.byref(p), C.byref(h)), what="foe_create")
    return h.value


def foe_destroy(ctx) -> None:
    if ctx:
        lib().foe_destroy(ctx)


def foe_step_size(ctx, bc: int = FOE_BC_SYMMETRIC, gamma: float = 0.8) -> tuple[float, float]:
    t, L = C.c_float(), C.c_double()
    _check(lib().foe_step_size(ctx, bc, gamma, C.byref(t), C.byref(L)), ctx, "foe_step_size")
    return t.value, L.value


def foe_denoise(ctx, y, x, H: int, W: int, ld: int, peak: float, opts: SolveOpts | None = None, stream=None,
                report: bool = False):
    o = (opts or SolveOpts()).c()
    rep = foe_report()
    _check(lib().foe_denoise(ctx, _ptr(y), _ptr(x), H, W, ld, peak, C.byref(o), _stream(stream),
                             C.byref(rep) if report else None), ctx, "foe_denoise")
    if report:
        return {"iters_done": rep.iters_done, "model_used": rep.model_used, "tau_used": rep.tau_used,
                "status": rep.status, "backtracks": rep.backtracks, "lipschitz_final": rep.lipschitz_final,
                "nonfinite": rep.nonfinite}
    return None


def foe_denoise_binned(ctx, y, x, H: int, W: int, ld: int, peak: float, opts: SolveOpts | None = None, stream=None,
                       report: bool = False):
    """The binning variant (3x3 bin sums, solve at 9 * peak, bilinear upscaling); arguments as foe_denoise."""
    o = (opts or SolveOpts()).c()
    rep = foe_report()
    _check(lib().foe_denoise_binned(ctx, _ptr(y), _ptr(x), H, W, ld, peak, C.byref(o), _stream(stream),
                                    C.byref(rep) if report else None), ctx, "foe_denoise_binned")
    if report:
        return {"iters_done": rep.iters_done, "model_used": rep.model_used, "tau_used": rep.tau_used,
                "status": rep.status, "backtracks": rep.backtracks, "lipschitz_final": rep.lipschitz_final,
                "nonfinite": rep.nonfinite}
    return None


def foe_step_log(ctx):
    """Trials of the last FOE_STEP_BACKTRACK solve: (tau per trial, accepted flag per trial) as numpy arrays."""
    import numpy as np
    n = lib().foe_step_log(ctx, None, None, 0)
    if n < 0:
        raise FoeError(FOE_EINVAL, "foe_step_log: invalid arguments")
    tau = np.zeros(n, dtype=np.float32)
    acc = np.zeros(n, dtype=np.uint8)
    if n:
        lib().foe_step_log(ctx, tau.ctypes.data_as(C.POINTER(C.c_float)), acc.ctypes.data_as(C.POINTER(C.c_ubyte)), n)
    return tau, acc.astype(bool)


def foe_denoise_static(ctx, y, x, H: int, W: int, ld: int, peak: float, opts: SolveOpts | None = None,
                       stream=None) -> None:
    """foe_denoise with the library's fixed device workspace instead of allocated memory (H * ld <= 2**20)."""
    o = (opts or SolveOpts()).c()
    _check(lib().foe_denoise_static(ctx, _ptr(y), _ptr(x), H, W, ld, peak, C.byref(o), _stream(stream)), ctx,
           "foe_denoise_static")


def foe_denoise_batch(ctx, descs: list[dict], opts: SolveOpts | None = None, stream=None) -> None:
    """descs: dicts with y, x (device buffers), H, W, ld, peak, iters, and optionally model (the image's own data
    term; without it the image takes opts.model)."""
    arr = (foe_image_desc * len(descs))()
    for j, d in enumerate(descs):
        m = d.get("model")
        arr[j] = foe_image_desc(_ptr(d["y"]), _ptr(d["x"]), d["H"], d["W"], d["ld"], d["peak"], d["iters"],
                                0 if m is None else 1, 0 if m is None else int(m))
    o = (opts or SolveOpts()).c()
    _check(lib().foe_denoise_batch(ctx, arr, len(descs), C.byref(o), _stream(stream)), ctx, "foe_denoise_batch")


def foe_iters_done(ctx, n: int = 1, stream=None) -> list[int]:
    """Iterations taken by each image of the last foe_denoise / foe_denoise_static / foe_denoise_batch solve (the
    stopping step, or the budget); synchronises the stream."""
    out = (C.c_int * n)()
    _check(lib().foe_iters_done(ctx, out, n, _stream(stream)), ctx, "foe_iters_done")
    return list(out)


def foe_energy_grad(ctx, u, data, H: int, W: int, ld: int, model: int, lam: float, bc: int = FOE_BC_SYMMETRIC,
                    prec: int = FOE_PREC_FP32, grad=None, energy: bool = True, stream=None):
    e = C.c_double()
    _check(lib().foe_energy_grad(ctx, _ptr(u), _ptr(data), H, W, ld, model, lam, bc, prec,
                                 C.byref(e) if energy else None, _ptr(grad), _stream(stream)), ctx, "foe_energy_grad")
    return e.value if energy else None


def foe_ipiano_step(ctx, u_hi, u_lo, delta, d, u_next_hi, H: int, W: int, ld: int, model: int, lam: float,
                    tau: float, gamma: float, bc: int = FOE_BC_SYMMETRIC, prec: int = FOE_PREC_FP32,
                    stream=None) -> None:
    _check(lib().foe_ipiano_step(ctx, _ptr(u_hi), _ptr(u_lo), _ptr(delta), _ptr(d), _ptr(u_next_hi), H, W, ld,
                                 model, lam, tau, gamma, bc, prec, _stream(stream)), ctx, "foe_ipiano_step")


def foe_anscombe(y, v, n: int, stream=None) -> None:
    _check(lib().foe_anscombe(_ptr(y), _ptr(v), n, _stream(stream)), what="foe_anscombe")


def foe_inverse(z, x, n: int, stream=None) -> None:
    _check(lib().foe_inverse(_ptr(z), _ptr(x), n, _stream(stream)), what="foe_inverse")


def foe_profile(ctx, enable: bool = True) -> None:
    _check(lib().foe_profile(ctx, 1 if enable else 0), ctx, "foe_profile")


def foe_profile_read(ctx) -> tuple[float, int, float]:
    """(summed step-loop device time in ms, step-kernel launches, pixel-iterations) since foe_profile(ctx, True)."""
    ms, n, px = C.c_double(), C.c_long(), C.c_double()
    _check(lib().foe_profile_read(ctx, C.byref(ms), C.byref(n), C.byref(px)), ctx, "foe_profile_read")
    return ms.value, n.value, px.value


def foe_mma_cost(m: int, n: int, a_in_tmem: bool = False, cta_pair: bool = False, issuers: int = 2,
                 count: int = 4096) -> float:
    """SM cycles per tcgen05.mma (kind::f16, K = 16) of an m x n shape; see include/foe.h."""
    out = C.c_double()
    _check(lib().foe_mma_cost(m, n, int(a_in_tmem), int(cta_pair), issuers, count, C.byref(out)), what="foe_mma_cost")
    return out.value


# ---- continuous-batching server ----
def foe_server_create(ctx, hbm_budget_bytes: int, max_active: int = 64, iters_per_tick: int = 10,
                      use_graphs: bool = True, opts: SolveOpts | None = None):
    cfg = foe_server_config(hbm_budget_bytes, max_active, iters_per_tick, 1 if use_graphs else 0,
                            (opts or SolveOpts()).c())
    h = C.c_void_p()
    _check(lib().foe_server_create(ctx, C.byref(cfg), C.byref(h)), ctx, "foe_server_create")
    return h.value


def foe_server_destroy(srv) -> None:
    if srv:
        lib().foe_server_destroy(srv)


def foe_server_submit(srv, y_host, x_host, H: int, W: int, peak: float, iters: int, y_pitch: int | None = None,
                      x_pitch: int | None = None, ctx=None) -> int:
    """y_host / x_host: host buffers (numpy arrays or torch CPU tensors, ideally page-locked)."""
    def addr(a):
        if isinstance(a, int):
            return a
        if hasattr(a, "data_ptr"):
            return int(a.data_ptr())
        return int(a.ctypes.data)
    rid = C.c_longlong()
    _check(lib().foe_server_submit(srv, addr(y_host), y_pitch or W, addr(x_host), x_pitch or W, H, W, peak, iters,
                                   C.byref(rid)), ctx, "foe_server_submit")
    return rid.value


def foe_server_tick(srv, ctx=None) -> int:
    n = C.c_int()
    _check(lib().foe_server_tick(srv, C.byref(n)), ctx, "foe_server_tick")
    return n.value


def foe_server_poll(srv, max_ids: int = 4096) -> list[int]:
    ids = (C.c_longlong * max_ids)()
    n = C.c_int()
    _check(lib().foe_server_poll(srv, ids, max_ids, C.byref(n)), what="foe_server_poll")
    return list(ids[:n.value])


def foe_server_get_stats(srv) -> dict:
    s = foe_server_stats()
    _check(lib().foe_server_get_stats(srv, C.byref(s)), what="foe_server_get_stats")
    return {k: getattr(s, k) for k, _ in foe_server_stats._fields_}


class foe_implicit_report(C.Structure):
    _fields_ = [("cg_iters", C.c_int), ("cg_relres", C.c_double), ("breakdowns", C.c_int)]


def foe_train_grad_implicit(ctx, clean, noisy, B: int, H: int, W: int, ld: int, opts: SolveOpts, dfilters, dlogalpha,
                            max_cg: int = 200, cg_tol: float = 1e-5, stream=None):
    """Loss and gradients by implicit differentiation at u^T (see include/foe.h); returns (loss, report dict)."""
    loss = C.c_double()
    rep = foe_implicit_report()
    o = opts.c()
    _check(lib().foe_train_grad_implicit(ctx, _ptr(clean), _ptr(noisy), B, H, W, ld, C.byref(o), int(max_cg),
                                         float(cg_tol), C.byref(loss), _ptr(dfilters), _ptr(dlogalpha), C.byref(rep),
                                         _stream(stream)), ctx, "foe_train_grad_implicit")
    return loss.value, {"cg_iters": rep.cg_iters, "cg_relres": rep.cg_relres, "breakdowns": rep.breakdowns}


def foe_train_step(ctx, clean, noisy, B: int, H: int, W: int, ld: int, opts: SolveOpts, dfilters, dlogalpha,
                   ckpt_every: int = 0, stream=None) -> float:
    """Loss and gradients of the unrolled solve (see include/foe.h); returns the loss."""
    loss = C.c_double()
    o = opts.c()
    _check(lib().foe_train_step(ctx, _ptr(clean), _ptr(noisy), B, H, W, ld, C.byref(o), ckpt_every, C.byref(loss),
                                _ptr(dfilters), _ptr(dlogalpha), _stream(stream)), ctx, "foe_train_step")
    return loss.value
