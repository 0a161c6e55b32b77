"""Writes tests/golden/oracle_512.json: FP64 oracle results for the 512x512 benchmark set.

The set is the paper's noise levels at the benchmark size: peaks {1, 2, 4, 8, 30} x {direct model,
Anscombe quadratic model, Anscombe I-divergence model}, 300 iPiano iterations, the seeded synthetic bank
and images.  For each
case it stores the oracle's PSNR against the clean image, a sample of output pixels, and a hash of
the inputs (so that a test can tell whether the generator still produces the same images).  It
calls only the oracle and the seeded input generator.

    python tests/golden/make_oracle_512.py
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1609_05722_gb300 import synth  # noqa: E402

H = W = 512
ITERS = 300
PEAKS = (1.0, 2.0, 4.0, 8.0, 30.0)
MODELS = ((0, "direct"), (1, "anscombe_l2"), (2, "anscombe_idiv"))
GAMMA = float(np.float32(0.8))
LAM = 1.0
NSAMPLE = 512


def case_inputs(pi, peak):
    seed = 1000 + 10 * pi
    clean = synth.clean_image(H, W, seed)
    y = synth.poisson_observation(clean, peak, seed + 5000)
    return clean * peak, y


def input_hash(k32, a32, y) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(k32).tobytes())
    h.update(np.ascontiguousarray(a32).tobytes())
    h.update(np.ascontiguousarray(y.astype(np.float32)).tobytes())
    return h.hexdigest()[:24]


def main():
    k, a = synth.filter_bank()
    k32, a32 = k.astype(np.float32), a.astype(np.float32)
    L = O.lipschitz(k32.astype(np.float64), a32.astype(np.float64), O.BC_SYMMETRIC, 512)
    tau = float(np.float32(0.99 * 2 * (1 - GAMMA) / (L + 2e-3)))
    rng = np.random.default_rng(12345)
    sample = rng.integers(0, H * W, NSAMPLE)
    out = {"H": H, "W": W, "iters": ITERS, "gamma": GAMMA, "lambda": LAM, "tau": tau, "bc": "symmetric",
           "sample_index": sample.tolist(), "cases": []}
    for pi, peak in enumerate(PEAKS):
        clean, y = case_inputs(pi, peak)
        for model, name in MODELS:
            pr = O.Problem(k32.astype(np.float64), a32.astype(np.float64), H, W, model=model, lam=LAM, tau=tau,
                           gamma=GAMMA)
            x, _ = pr.denoise(y, peak, ITERS)
            out["cases"].append({
                "peak": peak, "model": model, "name": name, "input_hash": input_hash(k32, a32, y),
                "psnr_oracle": O.psnr(x, clean, peak), "psnr_noisy": O.psnr(y, clean, peak),
                "x_sample": x.ravel()[sample].tolist(),
            })
            print(name, peak, out["cases"][-1]["psnr_noisy"], out["cases"][-1]["psnr_oracle"], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_512.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
