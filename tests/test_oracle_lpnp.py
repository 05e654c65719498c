"""Pins of the Algorithm 1 oracle.  CPU only."""
import numpy as np

import synthetic
from oracle import dsgnlm, forward, lpnp, problems

PSF = forward.gaussian_psf(1.0, 4)


def test_identity_denoiser_is_gradient_descent():
    # With W = I and C = R^n, u stays 0, v = x, and x <- x - mu grad f(x).
    # Compare with the same iteration written with an explicit dense A.
    from tests.test_oracle_forward import _dense_A
    H, W = 8, 10
    A = _dense_A(H, W, PSF)
    rng = np.random.default_rng(0)
    x0 = rng.uniform(0, 1, (H, W))
    y = rng.uniform(0, 1, (H // 2, W // 2))
    alpha, rho, iters = 1.0, 0.5, 12
    x, v, u, _ = lpnp.lpnp_solve(lambda x: forward.sr_grad(x, y, PSF), lambda z: z,
                                 x0, x0, np.zeros_like(x0), alpha, rho, iters, lpnp.NONE)
    mu = 1 / (alpha + rho)
    xd = x0.ravel().copy()
    for _ in range(iters):
        xd = xd - mu * (A.T @ (A @ xd - y.ravel()))
    np.testing.assert_allclose(x.ravel(), xd, atol=1e-13)
    np.testing.assert_allclose(u, 0, atol=1e-15)


def test_projection_sets():
    x = np.array([-0.5, 0.2, 1.7])
    np.testing.assert_array_equal(lpnp.project(x, lpnp.NONE), x)
    np.testing.assert_array_equal(lpnp.project(x, lpnp.NONNEG), [0, 0.2, 1.7])
    np.testing.assert_array_equal(lpnp.project(x, lpnp.BOX01), [0, 0.2, 1])


def test_residuals_decay_with_fixed_dsg_nlm():
    # fixed (F-DSG-NLM) W and alpha above the Lipschitz constant: linearized ADMM
    # converges, so the primal and dual residuals decay
    wl = synthetic.workload("sr64")
    inst = problems.sr_instance(wl, H=32, W=32)
    out = problems.solve_sr(wl, inst, iters=150, tol=1e-10)
    hist = out["hist"]
    assert hist[-1][0] < 1e-3 * hist[0][0]
    assert hist[-1][1] < 1e-3 * hist[0][1]
    x = out["x"]
    assert x.min() >= 0 and x.max() <= 1


def test_spi_solve_stays_in_box_and_settles():
    # h'' is unbounded at 0 (Sec. 4.2), so no convergence guarantee applies; the
    # iterates stay in [0, 1] and the dual residual drops over the first 50 steps
    wl = synthetic.workload("spi512")
    inst = problems.spi_instance(wl, H=24, W=20)
    out = problems.solve_spi(wl, inst, iters=50, tol=1e-10)
    x = out["x"]
    assert x.min() >= 0 and x.max() <= 1
    hist = out["hist"]
    assert hist[-1][1] < 0.1 * hist[0][1]


def test_one_adaptation_equals_fixed_w_from_first_input():
    # adapt_iters = 1: W is built once, from x^1 + u^0, and then frozen; the fixed
    # loop started from the same state with that W must give the same iterates
    wl = synthetic.workload("sr64")
    inst = problems.sr_instance(wl, H=16, W=20)
    y = inst["y"].astype(np.float64)
    g = forward.sr_guide(y)
    x0, v0, u0 = lpnp.initial_state(g)
    grad = lambda x: forward.sr_grad(x, y, PSF)
    mk = lambda z: (lambda zz, W=dsgnlm.build_w(z, 1, 2, 0.1, 1e-12, 10000)[0]: dsgnlm.denoise(W, zz))
    xa, va, ua, ha = lpnp.lpnp_solve_adaptive(grad, mk, x0, v0, u0, 1.0, 1.0, 6, 1, lpnp.BOX01)
    mu = 0.5
    x1 = np.clip(mu * (x0 + (v0 - u0) - grad(x0)), 0, 1)
    W1, _ = dsgnlm.build_w(x1 + u0, 1, 2, 0.1, 1e-12, 10000)
    xf, vf, uf, hf = lpnp.lpnp_solve(grad, lambda z: dsgnlm.denoise(W1, z), x0, v0, u0, 1.0, 1.0, 6, lpnp.BOX01)
    np.testing.assert_allclose(xa, xf, atol=1e-14)
    np.testing.assert_allclose(ua, uf, atol=1e-14)


def test_adaptive_loop_with_input_independent_denoiser_is_fixed_loop():
    wl = synthetic.workload("sr64")
    inst = problems.sr_instance(wl, H=12, W=12)
    y = inst["y"].astype(np.float64)
    g = forward.sr_guide(y)
    x0, v0, u0 = lpnp.initial_state(g)
    grad = lambda x: forward.sr_grad(x, y, PSF)
    W, _ = dsgnlm.build_w(g, 1, 2, 0.1, 1e-12, 10000)
    den = lambda z: dsgnlm.denoise(W, z)
    xa, _, ua, ha = lpnp.lpnp_solve_adaptive(grad, lambda z: den, x0, v0, u0, 1.0, 1.0, 7, 7, lpnp.BOX01)
    xf, _, uf, hf = lpnp.lpnp_solve(grad, den, x0, v0, u0, 1.0, 1.0, 7, lpnp.BOX01)
    np.testing.assert_array_equal(xa, xf)
    assert ha == hf


def test_adapt_then_freeze_converges():
    # the paper's F-DSG-NLM schedule: after the last adaptation W is fixed, so the
    # residuals decay (Sec. 4); A-DSG-NLM carries no such guarantee
    wl = synthetic.workload("sr64")
    inst = problems.sr_instance(wl, H=24, W=24)
    out = problems.solve_sr_adaptive(wl, inst, adapt_iters=5, iters=120, tol=1e-10)
    hist = out["hist"]
    assert len(out["infos"]) == 5
    assert hist[-1][0] < 1e-3 * hist[5][0]
    assert hist[-1][1] < 1e-3 * hist[5][1]
    assert out["x"].min() >= 0 and out["x"].max() <= 1


def test_conjugate_gradients_reach_the_direct_solution():
    rng = np.random.default_rng(4)
    B = rng.normal(size=(12, 12))
    M = B @ B.T + 0.5 * np.eye(12)
    b = rng.normal(size=12)
    x = lpnp.conjugate_gradients(lambda v: M @ v, b, np.zeros(12), 12)
    np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-8, atol=1e-10)


def test_standard_admm_with_identity_denoiser_is_proximal_point():
    # W = I, C = R^n: u stays 0, v = x, and x <- (A^T A + rho I)^{-1} (A^T y + rho x)
    from tests.test_oracle_forward import _dense_A_sym
    H, W = 8, 10
    A = _dense_A_sym(H, W, PSF)
    rng = np.random.default_rng(5)
    x0 = rng.uniform(0, 1, (H, W))
    y = rng.uniform(0, 1, (H // 2, W // 2))
    rho, iters = 0.7, 4
    x, v, u, _ = lpnp.admm_standard(lambda x: forward.sr_forward_sym(x, PSF), lambda r: forward.sr_adjoint_sym(r, PSF),
                                    y, lambda z: z, x0, x0, np.zeros_like(x0), rho, iters, H * W, lpnp.NONE)
    M = A.T @ A + rho * np.eye(H * W)
    xd = x0.ravel().copy()
    for _ in range(iters):
        xd = np.linalg.solve(M, A.T @ y.ravel() + rho * xd)
    np.testing.assert_allclose(x.ravel(), xd, atol=1e-9)
    np.testing.assert_allclose(u, 0, atol=1e-15)


def test_rms_literal_values():
    # rms(a) = sqrt(mean(a^2)): rms([3, 4]) = sqrt((9 + 16) / 2) = sqrt(12.5)
    assert lpnp.rms(np.array([3.0, 4.0])) == np.sqrt(12.5)
    assert lpnp.rms(np.full((5, 7), -0.25)) == 0.25
    assert lpnp.rms(np.zeros((3, 3))) == 0.0
    # the mean runs over every element of a 2-D image, not over rows
    assert abs(lpnp.rms(np.array([[1.0, 0.0], [0.0, 0.0]])) - 0.5) < 1e-15


def test_psnr_literal_values():
    # PSNR = 10 log10(1 / MSE), peak 1 over all pixels (reading of Sec. 4)
    ref = np.zeros((4, 4))
    assert abs(lpnp.psnr(np.full((4, 4), 0.1), ref) - 20.0) < 1e-12    # MSE 0.01
    assert abs(lpnp.psnr(np.full((4, 4), 0.01), ref) - 40.0) < 1e-12   # MSE 1e-4
    x = np.array([[0.5, 0.5], [0.5, 0.5]])
    y = np.array([[0.5, 0.5], [0.5, 0.7]])                              # MSE 0.04 / 4 = 0.01
    assert abs(lpnp.psnr(y, x) - 20.0) < 1e-12
    assert lpnp.psnr(x, x) == float("inf")
    assert abs(lpnp.psnr(x, y) - lpnp.psnr(y, x)) == 0.0


def test_residual_normalisation_two_pixels():
    # One step of Algorithm 1 on a 1x2 image worked out by hand (reading of Sec. 4,
    # Tables 2-3: RMS residuals, the dual one scaled by rho).  alpha = 1, rho = 2,
    # mu = 1/3, grad f = 0, x0 = v0 = (0.2, 0.6), u0 = 0:
    #   x1 = (1 x0 + 2 (v0 - u0)) / 3 = (0.2, 0.6);  z = x1 + u0 = (0.2, 0.6)
    #   v1 = W z with W = [[.5, .5], [.5, .5]]  ->  (0.4, 0.4)
    #   u1 = u0 + x1 - v1 = (-0.2, 0.2)
    #   primal = rms(x1 - v1) = 0.2;  dual = rho rms(v1 - v0) = 2 * 0.2 = 0.4
    #   PSNR against (0.2, 0.5): MSE = 0.01 / 2 -> 10 log10(200)
    x0 = np.array([[0.2, 0.6]])
    Wm = np.array([[0.5, 0.5], [0.5, 0.5]])
    x, v, u, hist = lpnp.lpnp_solve(lambda x: np.zeros_like(x), lambda z: (Wm @ z.ravel()).reshape(z.shape),
                                    x0, x0, np.zeros_like(x0), 1.0, 2.0, 1, lpnp.BOX01,
                                    np.array([[0.2, 0.5]]))
    np.testing.assert_allclose(x, [[0.2, 0.6]], atol=1e-15)
    np.testing.assert_allclose(v, [[0.4, 0.4]], atol=1e-15)
    np.testing.assert_allclose(u, [[-0.2, 0.2]], atol=1e-15)
    primal, dual, p = hist[0]
    assert abs(primal - 0.2) < 1e-15
    assert abs(dual - 0.4) < 1e-15
    assert abs(p - 10.0 * np.log10(200.0)) < 1e-12
