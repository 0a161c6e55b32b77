"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the benchmark.

This module only draws inputs.  It holds none of the denoiser's arithmetic: no
transform, no prior, no solver step.  Both sides of every parity check read the
same arrays from here.

Inputs stand in for data the paper uses but that is not available:

* clean test images (Sec. 5, eight natural images of 256x256 and 512x512) are
  replaced by a smooth gradient, six random disks/rectangles and a band-limited
  texture, min-max normalised to [0, 1];
* the learned FoE filters (Sec. 4, Fig. "filters": 48 filters of 7x7) are
  replaced by the 48 zero-mean atoms of the orthonormal 2-D DCT-7 basis (the
  constant atom removed, as in the paper's training set-up, Sec. 2.5.3), mixed by
  a seeded random orthogonal 48x48 matrix, so every filter is zero-mean with unit
  norm; weights alpha_i ~ U(0.5, 1.5);
* the Poisson observation follows Eq. (poissondistri): y_i ~ Poisson(peak * x_i).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

KSIZE = 7
NF = 48


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def clean_image(H: int, W: int, seed: int) -> np.ndarray:
    """Seeded clean image in [0, 1], float64, shape (H, W)."""
    rng = _rng(seed)
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    c0 = rng.uniform(0.0, 1.0)
    c1, c2 = rng.uniform(-0.5, 0.5, size=2)
    img = c0 + c1 * xx / W + c2 * yy / H
    side = min(H, W)
    for _ in range(6):
        cy = rng.uniform(0, H)
        cx = rng.uniform(0, W)
        size = rng.uniform(0.05, 0.25) * side
        val = rng.uniform(0.0, 1.0)
        if rng.uniform() < 0.5:
            mask = (yy - cy) ** 2 + (xx - cx) ** 2 <= size * size
        else:
            hy = size
            hx = rng.uniform(0.05, 0.25) * side
            mask = (np.abs(yy - cy) <= hy) & (np.abs(xx - cx) <= hx)
        img[mask] = val
    tex = np.zeros_like(img)
    for _ in range(8):
        wl = rng.uniform(4.0, 32.0)
        th = rng.uniform(0.0, math.pi)
        ph = rng.uniform(0.0, 2 * math.pi)
        tex += np.sin(2 * math.pi * (xx * math.cos(th) + yy * math.sin(th)) / wl + ph)
    img = img + (0.1 / 8.0) * tex
    lo, hi = img.min(), img.max()
    return (img - lo) / (hi - lo) if hi > lo else np.zeros_like(img)


def microscopy_tile(H: int, W: int, seed: int) -> np.ndarray:
    """Sparse bright Gaussian blobs on a dark background, max normalised to 1 (float64)."""
    rng = _rng(seed)
    img = np.full((H, W), rng.uniform(0.02, 0.05))
    nblobs = max(1, (H * W) // (64 * 64))
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    for _ in range(nblobs):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        s = rng.uniform(2.0, 8.0)
        a = rng.uniform(0.3, 1.0)
        r = max(1, int(4 * s))
        y0, y1 = max(0, int(cy) - r), min(H, int(cy) + r + 1)
        x0, x1 = max(0, int(cx) - r), min(W, int(cx) + r + 1)
        img[y0:y1, x0:x1] += a * np.exp(-((yy[y0:y1, x0:x1] - cy) ** 2 + (xx[y0:y1, x0:x1] - cx) ** 2) / (2 * s * s))
    return img / img.max()


def poisson_observation(clean: np.ndarray, peak: float, seed: int) -> np.ndarray:
    """y ~ Poisson(peak * clean), returned as float64 integer counts."""
    rng = _rng(seed)
    return rng.poisson(np.asarray(clean, dtype=np.float64) * float(peak)).astype(np.float64)


def _dct7_zero_mean_atoms() -> np.ndarray:
    """The 48 non-constant atoms of the orthonormal 2-D DCT-II basis of size 7x7."""
    n = np.arange(KSIZE)
    C = np.zeros((KSIZE, KSIZE))
    for k in range(KSIZE):
        s = math.sqrt(1.0 / KSIZE) if k == 0 else math.sqrt(2.0 / KSIZE)
        C[k] = s * np.cos(math.pi * (2 * n + 1) * k / (2 * KSIZE))
    atoms = []
    for k1 in range(KSIZE):
        for k2 in range(KSIZE):
            if k1 == 0 and k2 == 0:
                continue
            atoms.append(np.outer(C[k1], C[k2]))
    return np.stack(atoms)  # (48, 7, 7)


def filter_bank(nf: int = NF, seed: int = 7) -> tuple[np.ndarray, np.ndarray]:
    """Seeded synthetic FoE bank: (filters (nf, 7, 7) float64, alpha (nf,) float64).

    filters[i][a+3][b+3] is the convolution kernel k_i(a, b), a, b in -3..3.
    """
    if not 1 <= nf <= 48:
        raise ValueError("nf must be in 1..48")
    rng = _rng(seed)
    atoms = _dct7_zero_mean_atoms().reshape(48, KSIZE * KSIZE)
    G = rng.standard_normal((48, 48))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))[None, :]
    filt = (Q @ atoms)[:nf].reshape(nf, KSIZE, KSIZE)
    alpha = rng.uniform(0.5, 1.5, size=48)[:nf]
    return filt, alpha


@dataclass(frozen=True)
class ImageSpec:
    """One synthetic denoising problem: size, peak, iteration budget and seeds."""
    H: int
    W: int
    peak: float
    iters: int
    clean_seed: int
    noise_seed: int
    microscopy: bool = False


def make_problem(spec: ImageSpec) -> tuple[np.ndarray, np.ndarray]:
    """(clean scaled to [0, peak], noisy counts y), both float64."""
    if spec.microscopy:
        c = microscopy_tile(spec.H, spec.W, spec.clean_seed)
    else:
        c = clean_image(spec.H, spec.W, spec.clean_seed)
    return c * spec.peak, poisson_observation(c, spec.peak, spec.noise_seed)


def batched_uneven_specs(n: int = 64, seed: int = 3) -> list[ImageSpec]:
    """Mixed-size batch: sides from {128,...,1024} (H, W independent), peak log-U[1, 30], iters U{100..300}."""
    rng = _rng(seed)
    sides = [128, 256, 384, 512, 768, 1024]
    out = []
    for j in range(n):
        H = int(rng.choice(sides))
        W = int(rng.choice(sides))
        peak = float(math.exp(rng.uniform(math.log(1.0), math.log(30.0))))
        iters = int(rng.integers(100, 301))
        out.append(ImageSpec(H, W, peak, iters, 1000 + j, 5000 + j))
    return out


def serving_arrivals(n: int = 2000, rate_hz: float = 200.0, seed: int = 42,
                     micro_frac: float = 0.05) -> list[tuple[float, ImageSpec]]:
    """Poisson arrival stream: (arrival time in s, problem).  Sides log-U[128, 2048], 5% 4096^2 tiles."""
    rng = _rng(seed)
    t = 0.0
    out = []
    for j in range(n):
        t += float(rng.exponential(1.0 / rate_hz))
        if rng.uniform() < micro_frac:
            H = W = 4096
            peak = float(rng.uniform(1.0, 2.0))
            micro = True
        else:
            H = int(round(math.exp(rng.uniform(math.log(128), math.log(2048)))))
            W = int(round(math.exp(rng.uniform(math.log(128), math.log(2048)))))
            peak = float(math.exp(rng.uniform(math.log(1.0), math.log(30.0))))
            micro = False
        iters = 150 if peak < 5 else 100
        out.append((t, ImageSpec(H, W, peak, iters, 20000 + j, 60000 + j, micro)))
    return out
