"""FP64 oracle for DSG-NLM (Sec. 3 of the paper).  TEST INFRASTRUCTURE ONLY.

Every function follows one passage of Sec. 3 and is written for a reader to check
against it by eye; nothing here is blocked, fused or reordered.

Conventions (readings of passages the paper leaves open):

* pixels s, r of the image domain S are (row, column) pairs, flattened row-major;
* the search window Omega_s holds the r in S with |r - s|_inf <= N_s, clipped at the
  image border and never wrapped, which keeps r in Omega_s <=> s in Omega_r;
* patch pixels that fall outside the image read the guide extended by half-sample
  symmetric reflection (index -1 -> 0, H -> H-1), so the patch distance is
  symmetric in (s, r);
* the patch is N_p x N_p with N_p = 2 * patch_r + 1 and the window radius is
  N_s = search_r, so the hat of Eq. S1 is Lambda((s - r) / (search_r + 1));
* Eq. S2's one-shot normalisation is the first step of symmetric Sinkhorn-Knopp
  started from d = 1; ``sinkhorn(maxit=1)`` reproduces it and larger ``maxit``
  iterates it to a tolerance.  Eq. S3's "alpha" is 1/m, m the largest row sum.

Parity status: ``patch_distances`` and ``kernel_matrix`` are pinned by brute force
(``brute_force_kernel``) on tiny images; ``dsg_matrix`` by the Theorem IV.1
invariants (symmetric, doubly stochastic, spectrum in [0, 1]) and by closed forms
(constant guide, W = I cases); ``sinkhorn(maxit=1)`` + ``dsg_matrix`` by the
literal Algorithm 2 transcription ``alg2_literal``.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def sym_index(i, n: int):
    """Half-sample symmetric extension of index i into [0, n) (any integer i)."""
    m = np.mod(np.asarray(i), 2 * n)
    return np.where(m < n, m, 2 * n - 1 - m)


def extended(guide: np.ndarray, pad: int) -> np.ndarray:
    """Guide extended by ``pad`` pixels on every side by symmetric reflection."""
    H, W = guide.shape
    rows = sym_index(np.arange(-pad, H + pad), H)
    cols = sym_index(np.arange(-pad, W + pad), W)
    return guide[np.ix_(rows, cols)]


def hat(oy: int, ox: int, search_r: int) -> float:
    """Lambda((s - r) / (N_s + 1)) of Eq. S1: separable hat (1 - |a|)(1 - |b|)."""
    return (1.0 - abs(oy) / (search_r + 1.0)) * (1.0 - abs(ox) / (search_r + 1.0))


def window_offsets(search_r: int):
    """All offsets o = r - s of the (2 N_s + 1)^2 search window, row-major."""
    return [(oy, ox) for oy in range(-search_r, search_r + 1)
            for ox in range(-search_r, search_r + 1)]


def patch_distances(guide: np.ndarray, patch_r: int, oy: int, ox: int) -> np.ndarray:
    """||P_s - P_{s+o}||^2 for every s in S (Eq. NLM), as a direct sum over the
    N_p^2 patch pixels t: sum_t (g(s + t) - g(s + o + t))^2."""
    guide = np.asarray(guide, dtype=np.float64)
    H, W = guide.shape
    pad = patch_r + max(abs(oy), abs(ox))
    ge = extended(guide, pad)
    D = np.zeros((H, W))
    for ty in range(-patch_r, patch_r + 1):
        for tx in range(-patch_r, patch_r + 1):
            a = ge[pad + ty:pad + ty + H, pad + tx:pad + tx + W]
            b = ge[pad + ty + oy:pad + ty + oy + H, pad + tx + ox:pad + tx + ox + W]
            D += (a - b) ** 2
    return D


def kernel_matrix(guide: np.ndarray, patch_r: int, search_r: int, h: float) -> sp.csr_matrix:
    """K1 = [Lambda_{s,r} k_{s,r}] for r in Omega_s (Eq. NLM with sigma = h, Eq. S1).

    k_{s,r} = exp(-||P_s - P_r||^2 / (2 N_p^2 h^2)).  Sparse CSR, n x n, FP64.
    """
    guide = np.asarray(guide, dtype=np.float64)
    H, W = guide.shape
    n = H * W
    Np = 2 * patch_r + 1
    idx = np.arange(n).reshape(H, W)
    rows, cols, vals = [], [], []
    for oy, ox in window_offsets(search_r):
        i0, i1 = max(0, -oy), min(H, H - oy)
        j0, j1 = max(0, -ox), min(W, W - ox)
        if i0 >= i1 or j0 >= j1:
            continue
        D = patch_distances(guide, patch_r, oy, ox)
        w = hat(oy, ox, search_r) * np.exp(-D / (2.0 * Np * Np * h * h))
        rows.append(idx[i0:i1, j0:j1].ravel())
        cols.append(idx[i0 + oy:i1 + oy, j0 + ox:j1 + ox].ravel())
        vals.append(w[i0:i1, j0:j1].ravel())
    K1 = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(n, n))
    K1.sort_indices()
    return K1


def kernel_row(guide: np.ndarray, patch_r: int, search_r: int, h: float, s):
    """One row of K1: {r: K1(s, r)} for the r of Omega_s, computed pixel by pixel
    from the patch definition (for sampled checks on images too large for the
    sparse matrix)."""
    guide = np.asarray(guide, dtype=np.float64)
    H, W = guide.shape
    Np = 2 * patch_r + 1
    t = np.arange(-patch_r, patch_r + 1)
    ps = guide[np.ix_(sym_index(s[0] + t, H), sym_index(s[1] + t, W))]
    row = {}
    for oy, ox in window_offsets(search_r):
        r = (s[0] + oy, s[1] + ox)
        if not (0 <= r[0] < H and 0 <= r[1] < W):
            continue
        pr = guide[np.ix_(sym_index(r[0] + t, H), sym_index(r[1] + t, W))]
        D = float(np.sum((ps - pr) ** 2))
        row[r] = hat(oy, ox, search_r) * np.exp(-D / (2.0 * Np * Np * h * h))
    return row


def sinkhorn(K1: sp.spmatrix, tol: float, maxit: int):
    """Symmetric Sinkhorn-Knopp on K1 (Eq. S2 iterated).

    Starts from d = 1 and repeats d <- sqrt(d / (K1 d)) until the row sums of
    diag(d) K1 diag(d) are within ``tol`` of one (max-norm) or ``maxit`` updates
    were made.  The first update gives d = g^{-1/2} with g the row sums of K1,
    which is exactly Eq. S2.

    Returns (d, updates, residual history), the history holding
    max_s |d_s (K1 d)_s - 1| for d before any update and after each update.
    """
    d = np.ones(K1.shape[0])
    t = K1 @ d
    hist = [float(np.max(np.abs(d * t - 1.0)))]
    k = 0
    while k < maxit and hist[-1] > tol:
        d = np.sqrt(d / t)
        t = K1 @ d
        k += 1
        hist.append(float(np.max(np.abs(d * t - 1.0))))
    return d, k, hist


def dsg_matrix(K1: sp.spmatrix, d: np.ndarray):
    """W from K1 and the scaling d: S = diag(d) K1 diag(d); Eq. S3 with alpha = 1/m,
    m = max row sum of S: W = S/m, then w_ss <- 1 + w_ss - sum_r w_sr.

    Returns (W as CSR, m).
    """
    Dg = sp.diags(d)
    S = (Dg @ K1 @ Dg).tocsr()
    rowsum = np.asarray(S.sum(axis=1)).ravel()
    m = float(rowsum.max())
    W = S / m
    W = W + sp.diags(1.0 - np.asarray(W.sum(axis=1)).ravel())
    W = W.tocsr()
    W.sort_indices()
    return W, m


def build_w(guide, patch_r, search_r, h, tol, maxit):
    """DSG-NLM weight matrix: kernel, balance, closure.  Returns (W, info dict)."""
    K1 = kernel_matrix(guide, patch_r, search_r, h)
    d, k, hist = sinkhorn(K1, tol, maxit)
    W, m = dsg_matrix(K1, d)
    return W, dict(K1=K1, d=d, updates=k, hist=hist, m=m)


def denoise(W: sp.spmatrix, v: np.ndarray) -> np.ndarray:
    """DSG-NLM output W v (Sec. 3), v an image."""
    v = np.asarray(v, dtype=np.float64)
    return (W @ v.ravel()).reshape(v.shape)


# --------------------------------------------------------------------------------
# Independent literal forms, used as pins on tiny images only.
# --------------------------------------------------------------------------------

def _patch_dist_pointwise(guide, patch_r, s, r):
    H, W = guide.shape
    acc = 0.0
    for ty in range(-patch_r, patch_r + 1):
        for tx in range(-patch_r, patch_r + 1):
            a = guide[int(sym_index(s[0] + ty, H)), int(sym_index(s[1] + tx, W))]
            b = guide[int(sym_index(r[0] + ty, H)), int(sym_index(r[1] + tx, W))]
            acc += (float(a) - float(b)) ** 2
    return acc


def brute_force_kernel(guide, patch_r, search_r, h) -> np.ndarray:
    """Dense K1 by a literal loop over (s, r, patch pixel): the O(N_s^2 N_p^2)
    brute force of Sec. 4 (Table 1's slow column).  Tiny images only."""
    guide = np.asarray(guide, dtype=np.float64)
    H, W = guide.shape
    Np = 2 * patch_r + 1
    K = np.zeros((H * W, H * W))
    for si in range(H):
        for sj in range(W):
            for ri in range(H):
                for rj in range(W):
                    if abs(ri - si) > search_r or abs(rj - sj) > search_r:
                        continue
                    D = _patch_dist_pointwise(guide, patch_r, (si, sj), (ri, rj))
                    K[si * W + sj, ri * W + rj] = (
                        hat(ri - si, rj - sj, search_r)
                        * math.exp(-D / (2.0 * Np * Np * h * h)))
    return K


def alg2_literal(guide, vt, patch_r, search_r, h) -> np.ndarray:
    """Algorithm 2 (DSG-NLM filtering) transcribed as three aggregations over the
    pixels, recomputing Lambda k each time as the paper does.  The kernel is
    taken from ``guide`` (Algorithm 2 uses the input itself: pass guide = vt).
    Pure Python; tiny images only."""
    guide = np.asarray(guide, dtype=np.float64)
    vt = np.asarray(vt, dtype=np.float64)
    H, W = guide.shape
    Np = 2 * patch_r + 1
    pixels = [(i, j) for i in range(H) for j in range(W)]

    def omega(s):
        return [(i, j) for (i, j) in pixels
                if abs(i - s[0]) <= search_r and abs(j - s[1]) <= search_r]

    def lam_k(s, r):
        D = _patch_dist_pointwise(guide, patch_r, s, r)
        return hat(r[0] - s[0], r[1] - s[1], search_r) * math.exp(-D / (2.0 * Np * Np * h * h))

    g = {s: 0.0 for s in pixels}
    hh = {s: 0.0 for s in pixels}
    out = {s: 0.0 for s in pixels}
    m = 0.0
    # first aggregation: row sums of the hat-windowed kernel
    for s in pixels:
        for r in omega(s):
            g[s] += lam_k(s, r)
    # second aggregation: row sums after symmetric normalisation, and their maximum
    for s in pixels:
        delta = 0.0
        for r in omega(s):
            delta += (g[s] * g[r]) ** -0.5 * lam_k(s, r)
        m = max(m, delta)
    # third aggregation: scaled weights applied to the input, then the diagonal closure
    for s in pixels:
        for r in omega(s):
            w = (1.0 / m) * (g[s] * g[r]) ** -0.5 * lam_k(s, r)
            out[s] += w * vt[r]
            hh[s] += w
        out[s] += (1.0 - hh[s]) * vt[s]
    return np.array([[out[(i, j)] for j in range(W)] for i in range(H)])
