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
