"""Seeded synthetic inputs shared by the FP64 oracle, the tests and the benchmark.

This module holds no arithmetic of the restoration method: no blur, no decimation,
no patch distances, no kernel weights, no photon model.  It only draws the random
quantities the experiments need, all in FP64 from a seeded PCG64 stream and then
rounded once to FP32 so that every consumer sees bit-identical inputs:

* ``ground_truth``   piecewise-smooth test image in [0, 1] (ramp + shapes + texture),
                     standing in for the paper's test images (Sec. 4, Figs. 1 and 3),
                     which are not available;
* ``gaussian_noise`` i.i.d. N(0, sigma^2) samples for the additive noise of the
                     super-resolution model (Sec. 4.1, y = A x + n);
* ``photon_arrivals`` i.i.d. Exp(1) first-arrival variates, one per binary
                     sub-pixel of the single-photon sensor (Sec. 4.2).  A sub-pixel
                     with Poisson rate lam records a one iff its first arrival time
                     E ~ Exp(1) satisfies E < lam, so drawing E here and comparing it
                     with the rate elsewhere is the same experiment as thresholding
                     a Poisson count at one;
* ``batch_sides``    the uneven square sides of the batched workload.

The workload table (``WORKLOADS``) lists the five experiment configurations by
their sizes and parameters.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "ground_truth",
    "gaussian_noise",
    "photon_arrivals",
    "batch_sides",
    "WORKLOADS",
    "workload",
]


def _rng(seed: int, stream: int) -> np.random.Generator:
    # one independent PCG64 stream per (seed, purpose)
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def _periodic_gaussian_lowpass(field: np.ndarray, sigma: float) -> np.ndarray:
    """Low-pass a white field with a periodic Gaussian (texture synthesis only)."""
    H, W = field.shape
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    transfer = np.exp(-2.0 * (math.pi * sigma) ** 2 * (fy * fy + fx * fx))
    return np.real(np.fft.ifft2(np.fft.fft2(field) * transfer))


def ground_truth(H: int, W: int, n_shapes: int, texture: bool, seed: int) -> np.ndarray:
    """Synthetic piecewise-smooth grayscale image in [0, 1], FP32, shape (H, W).

    Recipe: a linear ramp 0.25 + 0.5 * p, where p is the projection of the pixel
    grid on a random direction theta ~ U[0, 2 pi) normalised to [0, 1]; then
    ``n_shapes`` shapes painted in order, each a rectangle or a disk with
    probability 1/2 and intensity U[0, 1] (rectangle sides U[H/16, H/4], disk
    radius U[H/32, H/8], centres uniform over the image); optionally a texture of
    white Gaussian noise low-passed by a periodic Gaussian of sigma 4 px and scaled
    to max-abs 0.05; finally clipped to [0, 1].
    """
    rng = _rng(seed, 0)
    ii, jj = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    theta = rng.uniform(0.0, 2.0 * math.pi)
    proj = ii * math.cos(theta) + jj * math.sin(theta)
    span = proj.max() - proj.min()
    proj = (proj - proj.min()) / (span if span > 0 else 1.0)
    img = 0.25 + 0.5 * proj
    side = float(min(H, W))
    for _ in range(n_shapes):
        is_rect = rng.uniform() < 0.5
        val = rng.uniform(0.0, 1.0)
        cy = rng.uniform(0.0, H)
        cx = rng.uniform(0.0, W)
        if is_rect:
            hh = rng.uniform(side / 16.0, side / 4.0)
            ww = rng.uniform(side / 16.0, side / 4.0)
            mask = (np.abs(ii - cy) <= hh / 2.0) & (np.abs(jj - cx) <= ww / 2.0)
        else:
            rad = rng.uniform(side / 32.0, side / 8.0)
            mask = (ii - cy) ** 2 + (jj - cx) ** 2 <= rad * rad
        img[mask] = val
    if texture:
        white = rng.standard_normal((H, W))
        tex = _periodic_gaussian_lowpass(white, 4.0)
        peak = np.abs(tex).max()
        if peak > 0:
            img = img + 0.05 * tex / peak
    img = np.clip(img, 0.0, 1.0)
    return img.astype(np.float32)


def gaussian_noise(shape, sigma: float, seed: int) -> np.ndarray:
    """I.i.d. N(0, sigma^2) samples, FP32."""
    rng = _rng(seed, 1)
    return (sigma * rng.standard_normal(shape)).astype(np.float32)


def photon_arrivals(shape, seed: int) -> np.ndarray:
    """I.i.d. Exp(1) first-arrival variates, FP32, one per binary sub-pixel."""
    rng = _rng(seed, 2)
    return rng.standard_exponential(shape).astype(np.float32)


def batch_sides(count: int, choices, seed: int) -> list[int]:
    """Square sides drawn uniformly from ``choices`` (uneven batch workload)."""
    rng = _rng(seed, 3)
    idx = rng.integers(0, len(choices), size=count)
    return [int(choices[i]) for i in idx]


# The five workloads: sizes, denoiser radii, bandwidth, tolerances and iteration
# counts.  "patch_r"/"search_r" are radii: a 7x7 patch is patch_r=3 and a 21x21
# search window is search_r=10.
WORKLOADS = {
    "sr64": dict(kind="sr", H=64, W=64, n_shapes=12, texture=False, seed=1001,
                 blur_sigma=1.0, blur_r=4, noise_sigma=0.02, patch_r=2, search_r=5,
                 h=0.1, tol=1e-8, iters=20, rho=1.0, alpha=1.0),
    "sr512": dict(kind="sr", H=512, W=512, n_shapes=40, texture=True, seed=1002,
                  blur_sigma=1.0, blur_r=4, noise_sigma=0.02, patch_r=3, search_r=10,
                  h=0.08, tol=1e-6, iters=30, rho=1.0, alpha=1.0),
    "spi512": dict(kind="spi", H=512, W=512, n_shapes=40, texture=True, seed=1003,
                   K_side=4, eta=4.0, spi_eps=1e-3, patch_r=3, search_r=10, h=0.1,
                   tol=1e-6, iters=50, rho=1.0, alpha=64.0),
    "batch64": dict(kind="sr", count=64, sides=(128, 256, 384, 512, 768, 1024),
                    n_shapes=40, texture=True, seed=1004, blur_sigma=1.0, blur_r=4,
                    noise_sigma=0.02, patch_r=3, search_r=10, h=0.08, tol=1e-6,
                    iters=30, rho=1.0, alpha=1.0),
    "unroll8x256": dict(kind="sr", count=8, H=256, W=256, n_shapes=40, texture=True,
                        seed=1005, blur_sigma=1.0, blur_r=4, noise_sigma=0.02,
                        patch_r=2, search_r=7, h=0.1, iters=10, rho=1.0, alpha=1.0),
}


def workload(name: str) -> dict:
    return dict(WORKLOADS[name])
