"""FP64 references for the derivatives of unrolled linearized PnP-ADMM.  TEST INFRASTRUCTURE ONLY.

The differentiable form fixes every discrete choice so that the output is a smooth
(piecewise smooth, through the box projection and the maximum m) function of its
inputs:
  * the DSG-NLM kernel K1 is built from the guide with bandwidth h (Eq. NLM, S1);
  * exactly T balancing passes d <- sqrt(d / K1 d) are made from d = 1 (no tolerance
    stop), then m = max_s d_s (K1 d)_s and the closure of Eq. S3 give W;
  * Algorithm 1 runs N iterations for 2x super-resolution from x = v = clip(guide),
    u = 0;
  * the loss is mean((x_N - x_true)^2).
The inputs that receive derivatives are the observation y, the guide, h and rho
(alpha, the blur and the radii are fixed).

Two independent references:
  * ``unrolled_loss`` in NumPy on the sparse oracle of ``dsgnlm`` / ``forward`` /
    ``lpnp`` (for central finite differences), and
  * ``torch_unrolled_loss``: the same function written with plain dense PyTorch FP64
    operations, differentiated by torch autograd.
Parity status: the two are checked against each other (tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np

from . import dsgnlm, forward, lpnp


def unrolled_loss(y, guide, h, rho, x_true, patch_r, search_r, T, N, alpha=1.0, psf=None, trace=None):
    """Loss of the unrolled solve (NumPy, FP64, sparse W).

    ``trace``, if a dict, receives the branches the loss took at its non-smooth
    points: "init" = sign(clip(guide) - guide) of the initial state, "argmax" =
    the first row of diag(d) K1 diag(d) whose sum is m, and "clamp" = the branch
    of Pi_C per pixel and iteration.  Two inputs with equal traces lie on one
    smooth piece of the loss, where central differences converge to the
    derivative (used to skip finite-difference points that straddle a kink)."""
    psf = forward.gaussian_psf(1.0, 4) if psf is None else psf
    guide = np.asarray(guide, np.float64)
    y = np.asarray(y, np.float64)
    K1 = dsgnlm.kernel_matrix(guide, patch_r, search_r, h)
    d, _, _ = dsgnlm.sinkhorn(K1, 0.0, T)
    W, _ = dsgnlm.dsg_matrix(K1, d)
    x0, v0, u0 = lpnp.initial_state(guide)
    clamps = [] if trace is not None else None
    x, _, _, _ = lpnp.lpnp_solve(lambda x: forward.sr_grad(x, y, psf), lambda z: dsgnlm.denoise(W, z),
                                 x0, v0, u0, alpha, rho, N, lpnp.BOX01, clamp_trace=clamps)
    if trace is not None:
        trace["init"] = np.sign(x0 - guide).astype(np.int8)
        trace["argmax"] = int(np.argmax(d * (K1 @ d)))
        trace["clamp"] = clamps
    return float(np.mean((x - np.asarray(x_true, np.float64)) ** 2))


def same_branches(a: dict, b: dict) -> bool:
    """True when two ``unrolled_loss`` traces took the same branch everywhere."""
    return (a["argmax"] == b["argmax"] and np.array_equal(a["init"], b["init"])
            and len(a["clamp"]) == len(b["clamp"])
            and all(np.array_equal(p, q) for p, q in zip(a["clamp"], b["clamp"])))


def fd_gradient(fn, x0, idx, eps):
    """Central difference of a scalar function along coordinate idx of array x0."""
    xp = np.array(x0, dtype=np.float64, copy=True)
    xm = np.array(x0, dtype=np.float64, copy=True)
    xp[idx] += eps
    xm[idx] -= eps
    return (fn(xp) - fn(xm)) / (2 * eps)


def torch_unrolled_loss(y, guide, h, rho, x_true, patch_r, search_r, T, N, alpha=1.0, sigma=1.0, blur_r=4):
    """The unrolled loss with dense PyTorch FP64 operations (for autograd).

    y, guide, h, rho may be torch tensors with requires_grad.  Dense n x n matrices:
    small images only.
    """
    import torch
    f64 = torch.float64
    guide = torch.as_tensor(guide, dtype=f64)
    y = torch.as_tensor(y, dtype=f64)
    h = torch.as_tensor(h, dtype=f64)
    rho = torch.as_tensor(rho, dtype=f64)
    x_true = torch.as_tensor(np.asarray(x_true, np.float64))
    H, W = guide.shape
    n = H * W
    Np = 2 * patch_r + 1
    # patches: reflected index grids (half-sample symmetric extension)
    rows = torch.as_tensor(dsgnlm.sym_index(np.arange(-patch_r, H + patch_r), H))
    cols = torch.as_tensor(dsgnlm.sym_index(np.arange(-patch_r, W + patch_r), W))
    ge = guide[rows][:, cols]
    patches = torch.stack([ge[a:a + H, b:b + W] for a in range(Np) for b in range(Np)], dim=-1)
    P = patches.reshape(n, Np * Np)
    D = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    ii = torch.arange(H).repeat_interleave(W)
    jj = torch.arange(W).repeat(H)
    dy = (ii[:, None] - ii[None, :]).abs()
    dx = (jj[:, None] - jj[None, :]).abs()
    inwin = (dy <= search_r) & (dx <= search_r)
    lam = (1 - dy.to(f64) / (search_r + 1)) * (1 - dx.to(f64) / (search_r + 1))
    K1 = torch.where(inwin, lam * torch.exp(-D / (2 * Np * Np * h * h)), torch.zeros((), dtype=f64))
    d = torch.ones(n, dtype=f64)
    for _ in range(T):
        d = torch.sqrt(d / (K1 @ d))
    S = d[:, None] * K1 * d[None, :]
    rs = S.sum(1)
    m = rs.max()
    Wm = S / m
    Wm = Wm + torch.diag(1 - Wm.sum(1))
    # forward model: periodic blur (dense circulant) + decimation
    a = torch.arange(-blur_r, blur_r + 1, dtype=f64)
    t1 = torch.exp(-a * a / (2 * sigma * sigma))
    t1 = t1 / t1.sum()
    psf = t1[:, None] * t1[None, :]
    A = torch.zeros((H // 2) * (W // 2), n, dtype=f64)
    for qi in range(H // 2):
        for qj in range(W // 2):
            for ai in range(-blur_r, blur_r + 1):
                for bj in range(-blur_r, blur_r + 1):
                    pi = (2 * qi - ai) % H
                    pj = (2 * qj - bj) % W
                    A[qi * (W // 2) + qj, pi * W + pj] += psf[ai + blur_r, bj + blur_r]
    yv = y.reshape(-1)
    x = torch.clamp(guide.reshape(-1), 0.0, 1.0)
    v = x.clone()
    u = torch.zeros(n, dtype=f64)
    mu = 1.0 / (alpha + rho)
    for _ in range(N):
        g = A.T @ (A @ x - yv)
        x = torch.clamp(mu * (alpha * x + rho * (v - u) - g), 0.0, 1.0)
        z = x + u
        v = Wm @ z
        u = z - v
    return ((x - x_true.reshape(-1)) ** 2).mean()
