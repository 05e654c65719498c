"""FP64 oracle for Algorithm 1 (linearized plug-and-play ADMM).  TEST INFRASTRUCTURE ONLY.

Algorithm 1, step by step, with mu = 1/(alpha + rho):
    x <- mu (alpha x + rho (v - u) - grad f(x))
    x <- Pi_C(x)
    v <- D(x + u)
    u <- u + (x - v)
D is DSG-NLM with a fixed W (the F-DSG-NLM variant of Sec. 4: W built once from a
guide and then frozen).  The initial values are x = v = clip(guide, 0, 1), u = 0.

Standard plug-and-play ADMM (the comparison of Sec. 4.1) replaces the linearized
x-update by the minimisation of f(x) + rho/2 ||x - (v - u)||^2: for the SR data
term, the linear system (A^T A + rho I) x = A^T y + rho (v - u), solved by
conjugate gradients (a fixed number of steps, started from the current x), then
the projection onto C.

The adaptive variants of Sec. 4 rebuild W from the denoiser input x + u: in every
iteration (A-DSG-NLM), or in the first ``adapt_iters`` iterations only, after
which the last W is kept (F-DSG-NLM with the paper's adapt-then-freeze schedule,
typically 15 iterations).

Residuals (Sec. 4, Tables 2-3, following Boyd et al.): primal ||x - v|| / sqrt(n)
and dual rho ||v^k - v^{k-1}|| / sqrt(n), reported as RMS values.  PSNR uses peak 1
over all pixels.

Parity status: conjugate gradients with n steps on an n-dimensional system equal a
direct solve; the standard loop with W = I and C = R^n is the proximal-point
iteration x <- (A^T A + rho I)^{-1}(A^T y + rho x), checked against dense solves.
The adaptive loop with one adaptation equals the fixed loop with W
built from x^1 + u^0, and with a denoiser that ignores its input it equals the
fixed loop.  With W = I and C = R^n the loop is gradient descent
x <- x - mu grad f(x); that case is pinned against an explicit dense-matrix
iteration.  With a fixed DSG-NLM W and alpha above the Lipschitz constant the
residuals decay (convergence of linearized ADMM, Sec. 2); that is checked as a
property.  End-to-end PSNR values are parity unpinned (the paper's test images
are not available).
"""
from __future__ import annotations

import math

import numpy as np

NONE, NONNEG, BOX01 = 0, 1, 2


def project(x: np.ndarray, constraint: int) -> np.ndarray:
    """Orthogonal projection Pi_C onto R^n, R^n_+ or [0, 1]^n (Sec. 2)."""
    if constraint == NONE:
        return x
    if constraint == NONNEG:
        return np.maximum(x, 0.0)
    if constraint == BOX01:
        return np.clip(x, 0.0, 1.0)
    raise ValueError(constraint)


def rms(a: np.ndarray) -> float:
    return float(np.sqrt(np.mean(np.asarray(a, dtype=np.float64) ** 2)))


def psnr(x: np.ndarray, ref: np.ndarray) -> float:
    mse = float(np.mean((np.asarray(x, np.float64) - np.asarray(ref, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)


def lpnp_solve(grad_f, denoise, x, v, u, alpha, rho, iters, constraint, x_true=None, clamp_trace=None):
    """Algorithm 1.  ``grad_f(x)`` and ``denoise(z)`` act on images.  Returns
    (x, v, u, history) with history[k] = (primal, dual, psnr or None).

    ``clamp_trace``, if a list, receives per iteration sign(Pi_C(x) - x) of the
    unprojected x-update: 0 where the projection is inactive, +1 / -1 where it
    raised / lowered the pixel.  It records which branch of Pi_C each pixel took
    and changes no arithmetic."""
    x = np.asarray(x, dtype=np.float64).copy()
    v = np.asarray(v, dtype=np.float64).copy()
    u = np.asarray(u, dtype=np.float64).copy()
    mu = 1.0 / (alpha + rho)
    hist = []
    for _ in range(iters):
        x = mu * (alpha * x + rho * (v - u) - grad_f(x))
        xp = project(x, constraint)
        if clamp_trace is not None:
            clamp_trace.append(np.sign(xp - x).astype(np.int8))
        x = xp
        v_prev = v
        v = denoise(x + u)
        u = u + (x - v)
        hist.append((rms(x - v), rho * rms(v - v_prev),
                     None if x_true is None else psnr(x, x_true)))
    return x, v, u, hist


def lpnp_solve_adaptive(grad_f, make_denoiser, x, v, u, alpha, rho, iters, adapt_iters, constraint,
                        x_true=None):
    """Algorithm 1 with W rebuilt from the denoiser input (Sec. 4): in iteration k <
    adapt_iters, ``make_denoiser(x + u)`` returns the denoiser built from x + u, which
    is then applied to x + u; later iterations keep the last one.  adapt_iters >= iters
    is A-DSG-NLM.  Returns (x, v, u, history) as lpnp_solve."""
    if adapt_iters < 1:
        raise ValueError("adapt_iters must be at least 1: W is built from x + u")
    x = np.asarray(x, dtype=np.float64).copy()
    v = np.asarray(v, dtype=np.float64).copy()
    u = np.asarray(u, dtype=np.float64).copy()
    mu = 1.0 / (alpha + rho)
    hist = []
    denoise = None
    for k in range(iters):
        x = mu * (alpha * x + rho * (v - u) - grad_f(x))
        x = project(x, constraint)
        z = x + u
        if k < adapt_iters:
            denoise = make_denoiser(z)
        v_prev = v
        v = denoise(z)
        u = u + (x - v)
        hist.append((rms(x - v), rho * rms(v - v_prev),
                     None if x_true is None else psnr(x, x_true)))
    return x, v, u, hist


def conjugate_gradients(apply_m, b, x, iters):
    """``iters`` steps of conjugate gradients for M x = b (M symmetric positive
    definite, given as a function), from x (Hestenes-Stiefel)."""
    x = np.asarray(x, dtype=np.float64).copy()
    r = b - apply_m(x)
    p = r.copy()
    rs = float(np.sum(r * r))
    for _ in range(iters):
        if rs == 0.0:
            break
        mp = apply_m(p)
        alpha = rs / float(np.sum(p * mp))
        x = x + alpha * p
        r = r - alpha * mp
        rs_new = float(np.sum(r * r))
        p = r + (rs_new / rs) * p
        rs = rs_new
    return x


def admm_standard(forward_op, adjoint_op, y, denoise, x, v, u, rho, iters, cg_iters, constraint, x_true=None):
    """Standard PnP-ADMM for f = 1/2 ||y - A x||^2: x <- Pi_C(CG solution of
    (A^T A + rho I) x = A^T y + rho (v - u), started from x); v <- D(x + u);
    u <- u + x - v.  Returns (x, v, u, history) as lpnp_solve."""
    x = np.asarray(x, dtype=np.float64).copy()
    v = np.asarray(v, dtype=np.float64).copy()
    u = np.asarray(u, dtype=np.float64).copy()
    aty = adjoint_op(np.asarray(y, dtype=np.float64))
    apply_m = lambda p: adjoint_op(forward_op(p)) + rho * p
    hist = []
    for _ in range(iters):
        x = conjugate_gradients(apply_m, aty + rho * (v - u), x, cg_iters)
        x = project(x, constraint)
        v_prev = v
        v = denoise(x + u)
        u = u + (x - v)
        hist.append((rms(x - v), rho * rms(v - v_prev),
                     None if x_true is None else psnr(x, x_true)))
    return x, v, u, hist


def initial_state(guide: np.ndarray):
    """x = v = clip(guide, 0, 1), u = 0."""
    x0 = np.clip(np.asarray(guide, dtype=np.float64), 0.0, 1.0)
    return x0.copy(), x0.copy(), np.zeros_like(x0)
