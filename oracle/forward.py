"""FP64 oracle for the two forward models of Sec. 4.  TEST INFRASTRUCTURE ONLY.

Super-resolution (Sec. 4.1): y = A x + n, A = periodic blur by a normalised
Gaussian h followed by keeping the pixels (2i, 2j); A^T = zero-filling at those
pixels followed by the adjoint blur (the same blur, h being symmetric).  The data
term is f = 1/2 ||y - A x||^2 (Eq. dataterm).  Its gradient is A^T (A x - y): the
paper prints A^T (y - A x), the negative gradient, and this file takes the
gradient.  The Lipschitz constant of the gradient is lambda_max(A^T A).

Single-photon imaging (Sec. 4.2): each pixel has K binary sub-pixels (a
sqrt(K) x sqrt(K) block), each seeing eta x / K photons on average; a sub-pixel
reads one iff its Poisson count is >= 1.  With K1_i ones and K0_i = K - K1_i zeros
in pixel i, f = sum_i h(x_i) (Eq. obj) with
h(t) = K0 eta t / K - K1 log(1 - exp(-eta t / K)) and h' as printed.  h' is
unbounded at t = 0, so the gradient is evaluated at max(x, eps).

Super-resolution with a symmetric boundary (the standard-vs-linearized comparison
of Sec. 4.1): the blur reads x extended by half-sample symmetric reflection,
(A_sym x)(q) = sum_t h(t) x(sym(2q - t)); its adjoint sends each term back to
sym(2q - t).

Guides (inputs of the fixed DSG-NLM, not defined by the paper): the SR guide is
a 2x Keys cubic (a = -0.5) interpolation of y with periodic wrap, low-resolution
sample j sitting at high-resolution 2j; the SPI guide is the per-pixel maximum-
likelihood intensity -(K/eta) log(1 - K1/K), clipped to [0, 1], smoothed by a
3x3 mean with symmetric reflection.

Parity status: ``sr_forward``/``sr_adjoint`` and their symmetric-boundary forms
pinned by the adjoint identity and by explicit dense matrices built from the
convolution definitions; ``sr_grad`` by
finite differences of ``sr_data``; ``sr_lipschitz`` by power iteration;
``spi_hprime`` by finite differences of ``spi_h`` and by h'(MLE) = 0;
``keys_up2`` by exact reproduction of quadratics; ``spi_observe``/``spi_counts``
by brute force against the Poisson definition on small blocks.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# Super-resolution
# ----------------------------------------------------------------------------

def gaussian_psf(sigma: float, r: int) -> np.ndarray:
    """(2r+1) x (2r+1) Gaussian exp(-(a^2 + b^2) / (2 sigma^2)), normalised to sum 1."""
    a = np.arange(-r, r + 1, dtype=np.float64)
    Y, X = np.meshgrid(a, a, indexing="ij")
    k = np.exp(-(Y * Y + X * X) / (2.0 * sigma * sigma))
    return k / k.sum()


def blur(x: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """Periodic convolution (h * x)(p) = sum_t h(t) x(p - t)."""
    x = np.asarray(x, dtype=np.float64)
    r = psf.shape[0] // 2
    out = np.zeros_like(x)
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            out += psf[a + r, b + r] * np.roll(x, shift=(a, b), axis=(0, 1))
    return out


def blur_adjoint(u: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """Adjoint of ``blur``: (h^T u)(p) = sum_t h(t) u(p + t)."""
    u = np.asarray(u, dtype=np.float64)
    r = psf.shape[0] // 2
    out = np.zeros_like(u)
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            out += psf[a + r, b + r] * np.roll(u, shift=(-a, -b), axis=(0, 1))
    return out


def sr_forward(x: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """A x: blur, then keep the pixels (2i, 2j)."""
    return blur(x, psf)[0::2, 0::2]


def sr_adjoint(r: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """A^T r: zero-fill r at the pixels (2i, 2j), then the adjoint blur."""
    h, w = r.shape
    up = np.zeros((2 * h, 2 * w))
    up[0::2, 0::2] = r
    return blur_adjoint(up, psf)


def sr_data(x, y, psf) -> float:
    """f(x) = 1/2 ||y - A x||^2 (Eq. dataterm)."""
    res = np.asarray(y, dtype=np.float64) - sr_forward(x, psf)
    return 0.5 * float(np.sum(res * res))


def sr_grad(x, y, psf) -> np.ndarray:
    """grad f(x) = A^T (A x - y)."""
    return sr_adjoint(sr_forward(x, psf) - np.asarray(y, dtype=np.float64), psf)


def sr_lipschitz(H: int, W: int, psf: np.ndarray) -> float:
    """lambda_max(A^T A) = lambda_max(A A^T).  A A^T is circulant on the
    low-resolution grid; its eigenvalues are the DFT of its first column."""
    delta = np.zeros((H // 2, W // 2))
    delta[0, 0] = 1.0
    col = sr_forward(sr_adjoint(delta, psf), psf)
    return float(np.max(np.real(np.fft.fft2(col))))


def _sym(i, n: int):
    """Half-sample symmetric reflection of index i into [0, n)."""
    m = np.mod(np.asarray(i), 2 * n)
    return np.where(m < n, m, 2 * n - 1 - m)


def sr_forward_sym(x: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """A_sym x: the blur of x extended by symmetric reflection, then the pixels (2i, 2j):
    (A_sym x)(q) = sum_t h(t) x(sym(2q - t))."""
    x = np.asarray(x, dtype=np.float64)
    H, W = x.shape
    r = psf.shape[0] // 2
    qi = 2 * np.arange(H // 2)
    qj = 2 * np.arange(W // 2)
    out = np.zeros((H // 2, W // 2))
    for a in range(-r, r + 1):
        rows = _sym(qi - a, H)
        for b in range(-r, r + 1):
            out += psf[a + r, b + r] * x[np.ix_(rows, _sym(qj - b, W))]
    return out


def sr_adjoint_sym(rlo: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """A_sym^T r: every term h(t) r(q) of A_sym goes back to pixel sym(2q - t)."""
    rlo = np.asarray(rlo, dtype=np.float64)
    h, w = rlo.shape
    H, W = 2 * h, 2 * w
    r = psf.shape[0] // 2
    out = np.zeros((H, W))
    qi = 2 * np.arange(h)
    qj = 2 * np.arange(w)
    for a in range(-r, r + 1):
        rows = _sym(qi - a, H)
        for b in range(-r, r + 1):
            cols = _sym(qj - b, W)
            np.add.at(out, (rows[:, None], cols[None, :]), psf[a + r, b + r] * rlo)
    return out


def sr_grad_sym(x, y, psf) -> np.ndarray:
    """grad f(x) = A_sym^T (A_sym x - y) for the symmetric-boundary model."""
    return sr_adjoint_sym(sr_forward_sym(x, psf) - np.asarray(y, dtype=np.float64), psf)


def sr_observe(x_true, noise, psf) -> np.ndarray:
    """Observation y = A x + n (Sec. 4.1), returned in FP64."""
    return sr_forward(x_true, psf) + np.asarray(noise, dtype=np.float64)


def keys_kernel(t, a: float = -0.5):
    """Keys cubic convolution kernel with parameter a."""
    t = np.abs(np.asarray(t, dtype=np.float64))
    out = np.zeros_like(t)
    near = t <= 1.0
    far = (t > 1.0) & (t < 2.0)
    out[near] = (a + 2.0) * t[near] ** 3 - (a + 3.0) * t[near] ** 2 + 1.0
    out[far] = a * t[far] ** 3 - 5.0 * a * t[far] ** 2 + 8.0 * a * t[far] - 4.0 * a
    return out


def keys_up2(y: np.ndarray) -> np.ndarray:
    """2x Keys cubic interpolation with periodic wrap; sample j sits at 2j."""
    y = np.asarray(y, dtype=np.float64)
    h, w = y.shape
    H, W = 2 * h, 2 * w

    def weights(n_out, n_in):
        M = np.zeros((n_out, n_in))
        for p in range(n_out):
            pos = p / 2.0
            for j in range(int(np.floor(pos)) - 2, int(np.floor(pos)) + 3):
                M[p, j % n_in] += keys_kernel(pos - j)
        return M

    return weights(H, h) @ y @ weights(W, w).T


def sr_guide(y) -> np.ndarray:
    """Guide of the SR experiments: Keys cubic 2x upsampling of y."""
    return keys_up2(y)


# ----------------------------------------------------------------------------
# Single-photon imaging
# ----------------------------------------------------------------------------

def spi_observe(x_true, arrivals, k_side: int, eta: float) -> np.ndarray:
    """Binary sub-pixel image: a sub-pixel of pixel i reads one iff its Poisson
    count with mean eta x_i / K is >= 1, i.e. iff its first arrival E ~ Exp(1)
    satisfies E < eta x_i / K.  Rate and comparison are taken in FP32, the
    precision of the stored arrivals and image, so every consumer makes the
    same decision.  Returns uint8 of shape (k_side H, k_side W)."""
    K = k_side * k_side
    x32 = np.asarray(x_true, dtype=np.float32)
    lam = (np.float32(eta) * x32) / np.float32(K)
    lam_sub = np.repeat(np.repeat(lam, k_side, axis=0), k_side, axis=1)
    return (np.asarray(arrivals, dtype=np.float32) < lam_sub).astype(np.uint8)


def spi_counts(bits: np.ndarray, k_side: int) -> np.ndarray:
    """K1_i: number of ones among the K = k_side^2 sub-pixels of pixel i."""
    Hs, Ws = bits.shape
    H, W = Hs // k_side, Ws // k_side
    return bits.reshape(H, k_side, W, k_side).astype(np.int64).sum(axis=(1, 3))


def spi_h(t, K0, K1, eta: float, K: int):
    """h(t) = -K0 log(exp(-eta t/K)) - K1 log(1 - exp(-eta t/K)) (Eq. obj)."""
    z = eta * np.asarray(t, dtype=np.float64) / K
    return K0 * z - K1 * np.log(-np.expm1(-z))


def spi_hprime(t, K0, K1, eta: float, K: int):
    """h'(t) = (eta/K) (K0 - K1 exp(-eta t/K) / (1 - exp(-eta t/K)))."""
    z = eta * np.asarray(t, dtype=np.float64) / K
    return (eta / K) * (K0 - K1 * np.exp(-z) / (-np.expm1(-z)))


def spi_grad(x, K1, eta: float, K: int, eps: float):
    """grad f(x)_i = h'(max(x_i, eps)) with K0 = K - K1."""
    K1 = np.asarray(K1, dtype=np.float64)
    return spi_hprime(np.maximum(np.asarray(x, dtype=np.float64), eps), K - K1, K1, eta, K)


def spi_data(x, K1, eta: float, K: int) -> float:
    K1 = np.asarray(K1, dtype=np.float64)
    return float(np.sum(spi_h(x, K - K1, K1, eta, K)))


def spi_mle(K1, eta: float, K: int) -> np.ndarray:
    """Per-pixel maximum-likelihood intensity -(K/eta) log(1 - K1/K), clipped to
    [0, 1] (K1 = K gives +inf, clipped to 1)."""
    K1 = np.asarray(K1, dtype=np.float64)
    with np.errstate(divide="ignore"):
        mle = -(K / eta) * np.log1p(-K1 / K)
    return np.clip(mle, 0.0, 1.0)


def box3_symmetric(img: np.ndarray) -> np.ndarray:
    """3x3 mean with half-sample symmetric reflection at the border."""
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape

    def refl(i, n):
        m = np.mod(i, 2 * n)
        return np.where(m < n, m, 2 * n - 1 - m)

    rows = refl(np.arange(-1, H + 1), H)
    cols = refl(np.arange(-1, W + 1), W)
    e = img[np.ix_(rows, cols)]
    out = np.zeros((H, W))
    for a in range(3):
        for b in range(3):
            out += e[a:a + H, b:b + W]
    return out / 9.0


def spi_guide(K1, eta: float, K: int) -> np.ndarray:
    return box3_symmetric(spi_mle(K1, eta, K))
