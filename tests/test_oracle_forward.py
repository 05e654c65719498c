"""Pins of the forward-model oracle (Sec. 4.1 super-resolution, Sec. 4.2 single-photon
imaging) and of the guide constructions.  CPU only."""
import math

import numpy as np
import pytest

from oracle import forward

PSF = forward.gaussian_psf(1.0, 4)


def _dense_A(H, W, psf):
    """A as an explicit matrix written from the definition:
    (A x)_q = sum_t h(t) x((2q - t) mod (H, W)), t over the taps [-r, r]^2
    (taps that wrap onto the same pixel add up)."""
    r = psf.shape[0] // 2
    A = np.zeros(((H // 2) * (W // 2), H * W))
    for qi in range(H // 2):
        for qj in range(W // 2):
            for a in range(-r, r + 1):
                for b in range(-r, r + 1):
                    pi = (2 * qi - a) % H
                    pj = (2 * qj - b) % W
                    A[qi * (W // 2) + qj, pi * W + pj] += psf[a + r, b + r]
    return A


def test_psf_normalised_and_symmetric():
    assert abs(PSF.sum() - 1) < 1e-15
    np.testing.assert_allclose(PSF, PSF[::-1, ::-1], atol=0)
    np.testing.assert_allclose(PSF, PSF.T, atol=0)
    # the centre tap of a sigma=1 Gaussian: 1 / (sum_a exp(-a^2/2))^2
    s = sum(math.exp(-a * a / 2) for a in range(-4, 5))
    assert abs(PSF[4, 4] - 1 / s ** 2) < 1e-15


def test_sr_forward_matches_dense_definition():
    H, W = 12, 10
    A = _dense_A(H, W, PSF)
    x = np.random.default_rng(0).uniform(0, 1, (H, W))
    np.testing.assert_allclose(forward.sr_forward(x, PSF).ravel(), A @ x.ravel(), atol=1e-14)
    r = np.random.default_rng(1).normal(size=(H // 2, W // 2))
    np.testing.assert_allclose(forward.sr_adjoint(r, PSF).ravel(), A.T @ r.ravel(), atol=1e-14)


def test_sr_adjoint_identity():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(32, 24))
    r = rng.normal(size=(16, 12))
    lhs = float(np.sum(forward.sr_forward(x, PSF) * r))
    rhs = float(np.sum(x * forward.sr_adjoint(r, PSF)))
    assert abs(lhs - rhs) < 1e-12 * max(1, abs(lhs))


def test_sr_gradient_finite_differences():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (10, 12))
    y = rng.uniform(0, 1, (5, 6))
    g = forward.sr_grad(x, y, PSF)
    eps = 1e-6
    for (i, j) in [(0, 0), (3, 7), (9, 11), (5, 2)]:
        e = np.zeros_like(x)
        e[i, j] = eps
        fd = (forward.sr_data(x + e, y, PSF) - forward.sr_data(x - e, y, PSF)) / (2 * eps)
        assert abs(fd - g[i, j]) < 1e-8


def test_sr_lipschitz_power_iteration():
    H, W = 16, 12
    L = forward.sr_lipschitz(H, W, PSF)
    v = np.random.default_rng(4).normal(size=(H, W))
    lam = 0.0
    for _ in range(500):
        w = forward.sr_adjoint(forward.sr_forward(v, PSF), PSF)
        lam = float(np.sum(w * v) / np.sum(v * v))
        v = w / np.linalg.norm(w)
    assert abs(lam - L) < 1e-9
    # the SR step size alpha = 1 exceeds the Lipschitz constant (about 1/4)
    assert 0.2 < L < 1.0


def test_keys_reproduces_quadratics_and_samples():
    # Keys' a = -0.5 cubic reproduces polynomials of degree <= 2 exactly
    h, w = 16, 14
    i = np.arange(h, dtype=np.float64)[:, None]
    j = np.arange(w, dtype=np.float64)[None, :]
    q = lambda a, b: 0.3 + 0.02 * a - 0.01 * b + 0.003 * a * a + 0.001 * a * b - 0.002 * b * b
    up = forward.keys_up2(q(i, j))
    # low-resolution samples are kept at the even pixels
    np.testing.assert_allclose(up[0::2, 0::2], q(i, j), atol=1e-14)
    # interior half-sample positions (two low-res samples from the wrap)
    P = np.arange(2 * h, dtype=np.float64)[:, None] / 2
    Q = np.arange(2 * w, dtype=np.float64)[None, :] / 2
    np.testing.assert_allclose(up[4:2 * h - 6, 4:2 * w - 6], q(P, Q)[4:2 * h - 6, 4:2 * w - 6],
                               atol=1e-13)
    # the half-sample weights are 9/16 and -1/16
    assert abs(forward.keys_kernel(0.5) - 9 / 16) < 1e-15
    assert abs(forward.keys_kernel(1.5) + 1 / 16) < 1e-15
    assert forward.keys_kernel(1.0) == 0 and forward.keys_kernel(2.0) == 0


def test_spi_hprime_finite_differences():
    eta, K = 4.0, 16
    for K1 in [0, 1, 7, 15, 16]:
        K0 = K - K1
        for t in [0.05, 0.3, 0.9]:
            eps = 1e-6
            fd = (forward.spi_h(t + eps, K0, K1, eta, K) - forward.spi_h(t - eps, K0, K1, eta, K)) / (2 * eps)
            assert abs(fd - forward.spi_hprime(t, K0, K1, eta, K)) < 1e-6 * max(1, abs(fd))


def test_spi_gradient_vanishes_at_mle():
    # for 0 < K1 < K the per-pixel likelihood is minimised at -(K/eta) log(1 - K1/K)
    eta, K = 4.0, 16
    for K1 in range(1, K):
        t = -(K / eta) * math.log(1 - K1 / K)
        assert abs(forward.spi_hprime(t, K - K1, K1, eta, K)) < 1e-12


def test_spi_observe_counts_brute_force():
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (3, 5)).astype(np.float32)
    arr = rng.standard_exponential((12, 20)).astype(np.float32)
    bits = forward.spi_observe(x, arr, 4, 4.0)
    counts = forward.spi_counts(bits, 4)
    for i in range(3):
        for j in range(5):
            lam = np.float32(np.float32(4.0) * x[i, j]) / np.float32(16)
            n = 0
            for a in range(4):
                for b in range(4):
                    one = arr[4 * i + a, 4 * j + b] < lam
                    assert bits[4 * i + a, 4 * j + b] == one
                    n += int(one)
            assert counts[i, j] == n


def test_spi_observe_frequency_matches_poisson():
    # P(Poisson(lam) >= 1) = 1 - exp(-lam)
    rng = np.random.default_rng(6)
    x = np.full((64, 64), 0.6, dtype=np.float32)
    arr = rng.standard_exponential((256, 256)).astype(np.float32)
    frac = forward.spi_observe(x, arr, 4, 4.0).mean()
    p = 1 - math.exp(-4.0 * 0.6 / 16)
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / arr.size)


def test_spi_guide_box_and_clip():
    K1 = np.array([[0, 16, 8], [1, 12, 3]])
    mle = forward.spi_mle(K1, 4.0, 16)
    assert mle[0, 0] == 0 and mle[0, 1] == 1
    assert abs(mle[0, 2] - min(1.0, -4 * math.log(0.5))) < 1e-15
    assert abs(mle[1, 0] - (-4 * math.log(15 / 16))) < 1e-15
    assert mle[1, 1] == 1  # -4 log(1/4) > 1 is clipped
    g = forward.box3_symmetric(np.full((4, 5), 0.3))
    np.testing.assert_allclose(g, 0.3, atol=1e-15)
    img = np.random.default_rng(7).uniform(0, 1, (4, 5))
    b = forward.box3_symmetric(img)
    # corner (0, 0): reflection repeats row 0 and column 0
    want = (img[0, 0] * 4 + img[0, 1] * 2 + img[1, 0] * 2 + img[1, 1]) / 9
    assert abs(b[0, 0] - want) < 1e-15


def _dense_A_sym(H, W, psf):
    """A_sym written from its definition: (A x)_q = sum_t h(t) x(sym(2q - t)), with
    sym the half-sample symmetric reflection (i -> -1 - i below 0, 2n - 1 - i above)."""
    def sym(i, n):
        while i < 0 or i >= n:
            i = -1 - i if i < 0 else 2 * n - 1 - i
        return i
    r = psf.shape[0] // 2
    A = np.zeros(((H // 2) * (W // 2), H * W))
    for qi in range(H // 2):
        for qj in range(W // 2):
            for a in range(-r, r + 1):
                for b in range(-r, r + 1):
                    A[qi * (W // 2) + qj, sym(2 * qi - a, H) * W + sym(2 * qj - b, W)] += psf[a + r, b + r]
    return A


@pytest.mark.parametrize("H,W", [(12, 10), (6, 4)])
def test_symmetric_sr_operator_matches_dense_definition(H, W):
    A = _dense_A_sym(H, W, PSF)
    x = np.random.default_rng(2).uniform(0, 1, (H, W))
    np.testing.assert_allclose(forward.sr_forward_sym(x, PSF).ravel(), A @ x.ravel(), atol=1e-14)
    r = np.random.default_rng(3).normal(size=(H // 2, W // 2))
    np.testing.assert_allclose(forward.sr_adjoint_sym(r, PSF).ravel(), A.T @ r.ravel(), atol=1e-14)
    # a constant image stays constant under the symmetric blur (the taps sum to 1)
    np.testing.assert_allclose(forward.sr_forward_sym(np.full((H, W), 0.3), PSF), 0.3, atol=1e-15)
