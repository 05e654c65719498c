"""GPU parity of the forward models, guides and Algorithm 1 against the FP64 oracle,
through the C ABI.  Integer outputs (bits, counts) must match exactly; FP32 outputs
within 1e-5 relative (the FP32 target), element-wise checks with tolerances
derived from the FP32 roundings of the sums involved."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import dsgnlm as odsg
from oracle import forward as ofw
from oracle import lpnp as olp
from oracle import problems
from tests.gpu_helpers import cuda, host, rel_l2

pytestmark = pytest.mark.gpu

PSF = ofw.gaussian_psf(1.0, 4)


@pytest.mark.parametrize("H,W", [(64, 64), (46, 70), (10, 12), (8, 8)])
def test_sr_observe_and_gradient(gpu_lib, H, W):
    from paper_1901_06110_gb300 import dsgnlm as D
    x = synthetic.ground_truth(H, W, 6, True, 77)
    noise = synthetic.gaussian_noise((H // 2, W // 2), 0.02, 77)
    y = host(D.lpnp_sr_observe(cuda(x), cuda(noise), 1.0, 4))
    want = ofw.sr_observe(x.astype(np.float64), noise.astype(np.float64), PSF)
    np.testing.assert_allclose(y, want, atol=2e-7 * 4, rtol=1e-6)
    yc = cuda(want.astype(np.float32))
    den = D.dsgnlm_create()
    xv = np.random.default_rng(1).uniform(0, 1, (H, W)).astype(np.float32)
    p = D.Problem("sr", den, cuda(xv), cuda(xv), cuda(xv), alpha=1.0, y=yc)
    g = host(D.lpnp_gradient(p, cuda(xv)))
    gw = ofw.sr_grad(xv.astype(np.float64), want.astype(np.float32).astype(np.float64), PSF)
    np.testing.assert_allclose(g, gw, atol=1e-6)


@pytest.mark.parametrize("h,w", [(32, 32), (23, 35), (1, 5)])
def test_sr_guide(gpu_lib, h, w):
    from paper_1901_06110_gb300 import dsgnlm as D
    y = np.random.default_rng(h).uniform(-0.1, 1.1, (h, w)).astype(np.float32)
    g = host(D.lpnp_sr_guide(cuda(y)))
    np.testing.assert_allclose(g, ofw.keys_up2(y.astype(np.float64)), atol=1e-6)


@pytest.mark.parametrize("H,W", [(64, 64), (33, 47)])
def test_spi_measurement_counts_guide_gradient(gpu_lib, H, W):
    from paper_1901_06110_gb300 import dsgnlm as D
    x = synthetic.ground_truth(H, W, 6, True, 88)
    arr = synthetic.photon_arrivals((4 * H, 4 * W), 88)
    bits = D.lpnp_spi_observe(cuda(x), cuda(arr), 4, 4.0)
    bits_o = ofw.spi_observe(x, arr, 4, 4.0)
    np.testing.assert_array_equal(host(bits), bits_o)
    counts = D.lpnp_spi_counts(bits, 4)
    counts_o = ofw.spi_counts(bits_o, 4)
    np.testing.assert_array_equal(host(counts).astype(np.int64), counts_o)
    g = host(D.lpnp_spi_guide(counts, 16, 4.0))
    np.testing.assert_allclose(g, ofw.spi_guide(counts_o, 4.0, 16), atol=2e-6)
    den = D.dsgnlm_create()
    xv = np.random.default_rng(3).uniform(0, 1, (H, W)).astype(np.float32)
    xv[0, :5] = 0.0  # below the floor eps
    p = D.Problem("spi", den, cuda(xv), cuda(xv), cuda(xv), alpha=64.0, counts=counts, K=16, eta=4.0,
                  spi_eps=1e-3)
    gr = host(D.lpnp_gradient(p, cuda(xv)))
    want = ofw.spi_grad(xv.astype(np.float64), counts_o, 4.0, 16, 1e-3)
    np.testing.assert_allclose(gr, want, rtol=2e-5, atol=1e-5)


def test_init_state(gpu_lib):
    from paper_1901_06110_gb300 import dsgnlm as D
    g = np.random.default_rng(5).uniform(-0.5, 1.5, (17, 19)).astype(np.float32)
    x, v, u = D.lpnp_init(cuda(g))
    x0, v0, u0 = olp.initial_state(g.astype(np.float64))
    np.testing.assert_array_equal(host(x), x0)
    np.testing.assert_array_equal(host(v), v0)
    np.testing.assert_array_equal(host(u), u0)


def _gpu_sr_solve(wl, y, iters, tol, maxit=10000, dtype="f32"):
    from paper_1901_06110_gb300 import dsgnlm as D
    yc = cuda(y)
    guide = D.lpnp_sr_guide(yc)
    den = D.dsgnlm_create(dtype)
    D.dsgnlm_build(den, guide, wl["patch_r"], wl["search_r"], wl["h"])
    st = D.dsgnlm_balance(den, tol, maxit)
    x, v, u = D.lpnp_init(guide)
    p = D.Problem("sr", den, x, v, u, alpha=wl["alpha"], y=yc, blur_sigma=wl["blur_sigma"],
                  blur_r=wl["blur_r"])
    hist = D.lpnp_solve(p, wl["rho"], iters, residuals=True)
    return dict(x=host(x), v=host(v), u=host(u), hist=hist, balance=st, guide=host(guide))


@pytest.mark.parametrize("H,W,rs", [(64, 64, 5), (46, 70, 4), (36, 98, 3), (10, 12, 2)])
def test_sr_solve_matches_oracle(gpu_lib, H, W, rs):
    wl = synthetic.workload("sr64")
    wl["search_r"] = rs
    inst = problems.sr_instance(wl, H=H, W=W)
    ref = problems.solve_sr(wl, inst, tol=1e-6)
    got = _gpu_sr_solve(wl, inst["y"], wl["iters"], 1e-6)
    assert got["balance"][0] == 0  # converged to 1e-6
    np.testing.assert_allclose(got["guide"], ref["guide"], atol=1e-6)
    for key in ("x", "v"):
        assert rel_l2(got[key], ref[key]) <= 1e-5, key
        np.testing.assert_allclose(got[key], ref[key], atol=2e-5)
    np.testing.assert_allclose(got["u"], ref["u"], atol=2e-5)
    # residual histories: RMS values down to ~1e-5, compared with an absolute floor
    for k, ((p, d), (po, do, _)) in enumerate(zip(got["hist"], ref["hist"])):
        assert abs(p - po) <= 1e-6 + 1e-3 * po, k
        assert abs(d - do) <= 1e-6 + 1e-3 * do, k


def test_sr_solve_paper_normalisation(gpu_lib):
    # the paper's own W (one normalisation step) inside Algorithm 1
    wl = synthetic.workload("sr64")
    inst = problems.sr_instance(wl, H=32, W=48)
    ref = problems.solve_sr(wl, inst, tol=0.0, maxit=1, iters=15)
    got = _gpu_sr_solve(wl, inst["y"], 15, 0.0, maxit=1)
    assert rel_l2(got["x"], ref["x"]) <= 1e-5


def test_spi_solve_matches_oracle(gpu_lib):
    from paper_1901_06110_gb300 import dsgnlm as D
    wl = synthetic.workload("spi512")
    wl["search_r"] = 5
    inst = problems.spi_instance(wl, H=40, W=56)
    iters = 10
    ref = problems.solve_spi(wl, inst, iters=iters, tol=1e-6)
    counts = cuda(inst["counts"].astype(np.uint8))
    guide = D.lpnp_spi_guide(counts, 16, wl["eta"])
    den = D.dsgnlm_create()
    D.dsgnlm_build(den, guide, wl["patch_r"], wl["search_r"], wl["h"])
    D.dsgnlm_balance(den, 1e-6, 10000)
    x, v, u = D.lpnp_init(guide)
    p = D.Problem("spi", den, x, v, u, alpha=wl["alpha"], counts=counts, K=16, eta=wl["eta"],
                  spi_eps=wl["spi_eps"])
    D.lpnp_solve(p, wl["rho"], iters)
    assert rel_l2(host(x), ref["x"]) <= 1e-5
    assert rel_l2(host(v), ref["v"]) <= 1e-5


def test_solve_rejects_bad_problems(gpu_lib):
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    den = D.dsgnlm_create()
    g = torch.rand((16, 16), device="cuda")
    y = torch.rand((8, 8), device="cuda")
    x, v, u = D.lpnp_init(g)
    p = D.Problem("sr", den, x, v, u, alpha=1.0, y=y)
    with pytest.raises(D.DsgnlmError) as e:
        D.lpnp_solve(p, 1.0, 3)
    assert e.value.status == _abi.NOT_BUILT
    D.dsgnlm_build(den, g, 1, 2, 0.1)
    with pytest.raises(D.DsgnlmError) as e:
        D.lpnp_solve(p, 1.0, 3)
    assert e.value.status == _abi.NOT_BALANCED
    D.dsgnlm_balance(den, 1e-6, 100)
    with pytest.raises(D.DsgnlmError) as e:
        D.lpnp_solve(p, -1.0, 3)
    assert e.value.status == _abi.EINVAL
    D.lpnp_solve(p, 1.0, 3)


def test_sr64_workload_as_specified(gpu_lib):
    """The 64x64 parity workload exactly as specified: 5x5 patches, 11x11 window,
    h = 0.1, balance to 1e-8, 20 iterations, through the benchmark's pipeline.

    1e-8 lies below the FP32 floor of the stored scaling d (about 1e-7), so the
    balance may end STALLED with the achieved residual reported (reading of the
    FP32 Sinkhorn floor); W stays doubly stochastic through the closure of Eq. S3,
    and x, v must still match the oracle balanced to 1e-8 within 1e-5 relative
    (Eq. S2 iterated, Eq. S3, Algorithm 1)."""
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    from paper_1901_06110_gb300 import pipeline
    wl = synthetic.workload("sr64")
    assert (wl["tol"], wl["iters"], wl["patch_r"], wl["search_r"]) == (1e-8, 20, 2, 5)
    inst = problems.sr_instance(wl)
    ref = problems.solve_sr(wl, inst)
    assert ref["info"]["hist"][-1] <= 1e-8  # the oracle itself reaches the tolerance in FP64
    solver = pipeline.Solver(64, 64, pipeline.Params.from_workload(wl))
    hist = solver.run(cuda(inst["y"]), residuals=True)
    torch.cuda.synchronize()
    st, updates, resid = solver.balance
    assert st in (_abi.OK, _abi.STALLED), solver.balance
    assert np.isfinite(resid) and resid <= 1e-6 and updates >= 1
    if st == _abi.OK:
        assert resid <= 1e-8
    ones = torch.ones((64, 64), device="cuda")
    np.testing.assert_allclose(host(D.dsgnlm_apply(solver.den, ones)), 1.0, atol=1e-6)
    for key, t in (("x", solver.x), ("v", solver.v)):
        assert rel_l2(host(t), ref[key]) <= 1e-5, key
    np.testing.assert_allclose(host(solver.u), ref["u"], atol=2e-5)
    for k, ((p, d), (po, do, _)) in enumerate(zip(hist, ref["hist"])):
        assert abs(p - po) <= 1e-6 + 1e-3 * po, k
        assert abs(d - do) <= 1e-6 + 1e-3 * do, k
    solver.close()
