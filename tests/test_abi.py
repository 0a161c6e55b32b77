"""C ABI checks that need no GPU: the library builds for sm_103a, loads, exports every entry point
that include/foe.h declares, and its host-only logic (argument checks, step size) is right."""
import ctypes as C
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_1609_05722_gb300 import build as B
from paper_1609_05722_gb300 import foe as F

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "foe.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return F.lib()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"FOE_API\s+[\w\s\*]*?\b(foe_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("foe_create", "foe_destroy", "foe_denoise", "foe_denoise_batch", "foe_denoise_binned",
                     "foe_train_grad_implicit", "foe_energy_grad",
                     "foe_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert F.foe_status_string(F.FOE_OK) == "ok"
    assert F.foe_status_string(F.FOE_EINVAL) == "invalid argument"
    assert F.foe_status_string(99) == "unknown status"


def test_default_opts(lib):
    o = F.foe_default_opts()
    assert (o.model, o.iters, o.bc, o.prec, o.step) == (F.FOE_MODEL_AUTO, 300, F.FOE_BC_SYMMETRIC, F.FOE_PREC_BF16,
                                                       F.FOE_STEP_FIXED)
    assert o.lam == 1.0 and o.gamma == pytest.approx(0.8) and o.tau == 0.0


@pytest.mark.parametrize("bc", [F.FOE_BC_SYMMETRIC, F.FOE_BC_ZERO])
def test_lipschitz_bound_matches_oracle(lib, bank, bc):
    # two independent evaluations of 2 kappa max_w sum_i alpha_i |k_i^(w)|^2 on the 512 grid
    k, a = bank
    k32, a32 = k.astype(np.float32), a.astype(np.float32)
    got = F.foe_prior_lipschitz(k32, a32, bc)
    ref = O.lipschitz(k32.astype(np.float64), a32.astype(np.float64), bc, 512)
    assert got == pytest.approx(ref, rel=1e-10)


def test_invalid_arguments_are_rejected_on_the_host(lib, bank):
    k, a = bank
    # bad priors never reach the device
    p = F.foe_prior(0, 7, None, None)
    h = C.c_void_p()
    assert lib.foe_create(C.byref(p), C.byref(h)) == F.FOE_EINVAL
    with pytest.raises(F.FoeError):
        F.foe_prior_lipschitz(k[:, :6, :6], a)
    bad_alpha = a.copy()
    bad_alpha[3] = -1.0
    with pytest.raises(F.FoeError):
        F.foe_prior_lipschitz(k, bad_alpha)
    # calls without a context
    o = F.SolveOpts().c()
    assert lib.foe_denoise(None, 16, 16, 64, 64, 64, 4.0, C.byref(o), None, None) == F.FOE_EINVAL
    assert lib.foe_energy_grad(None, 16, 16, 64, 64, 64, 1, 1.0, 0, 0, None, None, None) == F.FOE_EINVAL
    assert lib.foe_anscombe(None, None, -1, None) == F.FOE_EINVAL


@pytest.mark.parametrize("args", [(100, 64, 0, 0, 2, 16), (128, 40, 0, 0, 2, 16), (64, 60, 0, 0, 2, 16),
                                  (64, 64, 1, 0, 2, 16), (128, 256, 1, 0, 2, 16), (128, 64, 0, 1, 2, 16),
                                  (256, 64, 1, 1, 2, 16), (128, 64, 0, 0, 3, 16), (128, 64, 0, 0, 2, 0)])
def test_mma_cost_rejects_bad_shapes_on_the_host(lib, args):
    # checked before any device call, so this runs without a GPU
    out = C.c_double(-1.0)
    assert lib.foe_mma_cost(*args, C.byref(out)) == F.FOE_EINVAL
    assert out.value == -1.0


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "foe.h"

int main(void)
{
    foe_solve_opts o;
    double out = -1.0;
    if (foe_default_opts(&o) != FOE_OK) return 1;
    if (o.iters != 300 || o.model != FOE_MODEL_AUTO || o.prec != FOE_PREC_BF16) return 2;
    if (strcmp(foe_status_string(FOE_EINVAL), "invalid argument") != 0) return 3;
    if (foe_mma_cost(100, 64, 0, 0, 2, 16, &out) != FOE_EINVAL || out != -1.0) return 4;
    puts("ok");
    return 0;
}
"""


def test_header_is_plain_c_and_links(lib, tmp_path):
    # the boundary is a C ABI: a C99 program includes the header with every warning an error, links against the
    # library and calls its host-only entry points (no GPU needed)
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src, exe = tmp_path / "client.c", tmp_path / "client"
    src.write_text(C_CLIENT)
    libdir = os.path.dirname(B.LIB)
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", f"-I{os.path.dirname(HEADER)}", str(src),
           f"-L{libdir}", "-lfoe", f"-Wl,-rpath,{libdir}", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
