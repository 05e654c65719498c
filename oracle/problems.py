"""FP64 oracle: the experiments of Sec. 4 assembled end to end.  TEST INFRASTRUCTURE ONLY.

Builds a synthetic instance (ground truth from ``synthetic``), its measurements
with the oracle's own forward models, and runs Algorithm 1 with a fixed DSG-NLM W.
The measurements handed to the CUDA path in the tests are the FP32 roundings of
the values made here, so both sides start from identical inputs.
"""
from __future__ import annotations

import numpy as np

import synthetic
from . import dsgnlm, forward, lpnp


def sr_instance(wl: dict, H: int | None = None, W: int | None = None, seed: int | None = None):
    """Ground truth, FP32 observation y = A x + n and the FP32 noise used."""
    H = wl["H"] if H is None else H
    W = wl["W"] if W is None else W
    seed = wl["seed"] if seed is None else seed
    x_true = synthetic.ground_truth(H, W, wl["n_shapes"], wl["texture"], seed)
    noise = synthetic.gaussian_noise((H // 2, W // 2), wl["noise_sigma"], seed)
    psf = forward.gaussian_psf(wl["blur_sigma"], wl["blur_r"])
    y = forward.sr_observe(x_true, noise, psf).astype(np.float32)
    return dict(x_true=x_true, noise=noise, y=y, psf=psf)


def spi_instance(wl: dict, H: int | None = None, W: int | None = None, seed: int | None = None):
    """Ground truth, FP32 arrivals, the binary sub-pixel image and the counts."""
    H = wl["H"] if H is None else H
    W = wl["W"] if W is None else W
    seed = wl["seed"] if seed is None else seed
    ks = wl["K_side"]
    x_true = synthetic.ground_truth(H, W, wl["n_shapes"], wl["texture"], seed)
    arrivals = synthetic.photon_arrivals((ks * H, ks * W), seed)
    bits = forward.spi_observe(x_true, arrivals, ks, wl["eta"])
    counts = forward.spi_counts(bits, ks)
    return dict(x_true=x_true, arrivals=arrivals, bits=bits, counts=counts)


def solve_sr(wl: dict, inst: dict, iters: int | None = None, tol: float | None = None,
             maxit: int = 10000, guide=None):
    """Algorithm 1 for 2x super-resolution with F-DSG-NLM built from the guide."""
    psf = inst["psf"]
    y = inst["y"].astype(np.float64)
    g = forward.sr_guide(y) if guide is None else np.asarray(guide, np.float64)
    W, info = dsgnlm.build_w(g, wl["patch_r"], wl["search_r"], wl["h"],
                             wl["tol"] if tol is None else tol, maxit)
    x0, v0, u0 = lpnp.initial_state(g)
    out = lpnp.lpnp_solve(lambda x: forward.sr_grad(x, y, psf),
                          lambda z: dsgnlm.denoise(W, z), x0, v0, u0,
                          wl["alpha"], wl["rho"], wl["iters"] if iters is None else iters,
                          lpnp.BOX01, inst["x_true"])
    return dict(guide=g, W=W, info=info, x=out[0], v=out[1], u=out[2], hist=out[3])


def solve_spi(wl: dict, inst: dict, iters: int | None = None, tol: float | None = None,
              maxit: int = 10000, guide=None):
    """Algorithm 1 for single-photon imaging with F-DSG-NLM built from the guide."""
    K = wl["K_side"] ** 2
    counts = inst["counts"]
    g = forward.spi_guide(counts, wl["eta"], K) if guide is None else np.asarray(guide, np.float64)
    W, info = dsgnlm.build_w(g, wl["patch_r"], wl["search_r"], wl["h"],
                             wl["tol"] if tol is None else tol, maxit)
    x0, v0, u0 = lpnp.initial_state(g)
    out = lpnp.lpnp_solve(lambda x: forward.spi_grad(x, counts, wl["eta"], K, wl["spi_eps"]),
                          lambda z: dsgnlm.denoise(W, z), x0, v0, u0,
                          wl["alpha"], wl["rho"], wl["iters"] if iters is None else iters,
                          lpnp.BOX01, inst["x_true"])
    return dict(guide=g, W=W, info=info, x=out[0], v=out[1], u=out[2], hist=out[3])


def solve_sr_adaptive(wl: dict, inst: dict, adapt_iters: int, iters: int | None = None,
                      tol: float | None = None, maxit: int = 10000):
    """Algorithm 1 for 2x super-resolution with W rebuilt from x + u in the first
    adapt_iters iterations (A-DSG-NLM when adapt_iters >= iters, the paper's
    F-DSG-NLM schedule otherwise).  The initial state comes from the bicubic guide."""
    psf = inst["psf"]
    y = inst["y"].astype(np.float64)
    g = forward.sr_guide(y)
    tol = wl["tol"] if tol is None else tol
    infos = []

    x0, v0, u0 = lpnp.initial_state(g)
    return _adaptive(wl, lambda x: forward.sr_grad(x, y, psf), g, x0, v0, u0, inst["x_true"], adapt_iters, iters,
                     tol, maxit)


def solve_spi_adaptive(wl: dict, inst: dict, adapt_iters: int, iters: int | None = None,
                       tol: float | None = None, maxit: int = 10000):
    """Algorithm 1 for single-photon imaging with W rebuilt from x + u in the first
    adapt_iters iterations.  The initial state comes from the MLE guide."""
    K = wl["K_side"] ** 2
    counts = inst["counts"]
    g = forward.spi_guide(counts, wl["eta"], K)
    x0, v0, u0 = lpnp.initial_state(g)
    grad = lambda x: forward.spi_grad(x, counts, wl["eta"], K, wl["spi_eps"])
    return _adaptive(wl, grad, g, x0, v0, u0, inst["x_true"], adapt_iters, iters, tol, maxit)


def _adaptive(wl, grad, g, x0, v0, u0, x_true, adapt_iters, iters, tol, maxit):
    tol = wl["tol"] if tol is None else tol
    infos, mats = [], []

    def make_denoiser(z):
        W, info = dsgnlm.build_w(z, wl["patch_r"], wl["search_r"], wl["h"], tol, maxit)
        infos.append(info)
        mats.append(W)
        return lambda zz: dsgnlm.denoise(W, zz)

    out = lpnp.lpnp_solve_adaptive(grad, make_denoiser, x0, v0, u0, wl["alpha"], wl["rho"],
                                   wl["iters"] if iters is None else iters, adapt_iters, lpnp.BOX01, x_true)
    return dict(guide=g, infos=infos, W_last=mats[-1], x=out[0], v=out[1], u=out[2], hist=out[3])


def sr_instance_sym(wl: dict, H: int | None = None, W: int | None = None, seed: int | None = None):
    """Ground truth and FP32 observation y = A_sym x + n for the symmetric-boundary model."""
    H = wl["H"] if H is None else H
    W = wl["W"] if W is None else W
    seed = wl["seed"] if seed is None else seed
    x_true = synthetic.ground_truth(H, W, wl["n_shapes"], wl["texture"], seed)
    noise = synthetic.gaussian_noise((H // 2, W // 2), wl["noise_sigma"], seed)
    psf = forward.gaussian_psf(wl["blur_sigma"], wl["blur_r"])
    y = (forward.sr_forward_sym(x_true, psf) + noise.astype(np.float64)).astype(np.float32)
    return dict(x_true=x_true, noise=noise, y=y, psf=psf)


def solve_sr_sym(wl: dict, inst: dict, iters: int | None = None, tol: float | None = None, maxit: int = 10000,
                 standard_cg_iters: int = 0):
    """2x SR with the symmetric-boundary model and F-DSG-NLM from the bicubic guide:
    linearized PnP-ADMM (Algorithm 1), or with standard_cg_iters > 0 standard PnP-ADMM
    whose x-update takes that many conjugate-gradient steps."""
    psf = inst["psf"]
    y = inst["y"].astype(np.float64)
    g = forward.sr_guide(y)
    W, info = dsgnlm.build_w(g, wl["patch_r"], wl["search_r"], wl["h"],
                             wl["tol"] if tol is None else tol, maxit)
    x0, v0, u0 = lpnp.initial_state(g)
    n = wl["iters"] if iters is None else iters
    den = lambda z: dsgnlm.denoise(W, z)
    if standard_cg_iters > 0:
        out = lpnp.admm_standard(lambda x: forward.sr_forward_sym(x, psf), lambda r: forward.sr_adjoint_sym(r, psf),
                                 y, den, x0, v0, u0, wl["rho"], n, standard_cg_iters, lpnp.BOX01, inst["x_true"])
    else:
        out = lpnp.lpnp_solve(lambda x: forward.sr_grad_sym(x, y, psf), den, x0, v0, u0, wl["alpha"], wl["rho"], n,
                              lpnp.BOX01, inst["x_true"])
    return dict(guide=g, W=W, info=info, x=out[0], v=out[1], u=out[2], hist=out[3])
