"""The symmetric-boundary SR model and standard PnP-ADMM with a conjugate-gradient
x-update (the standard-vs-linearized comparison of Sec. 4.1) against the FP64
oracle: the observation and gradient element by element, the linearized and the
standard solves at 1e-5 relative."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import forward as ofw
from oracle import problems
from tests.gpu_helpers import cuda, host, rel_l2

pytestmark = pytest.mark.gpu

PSF = ofw.gaussian_psf(1.0, 4)


@pytest.mark.parametrize("H,W", [(64, 64), (46, 70), (8, 12)])
def test_symmetric_observation_and_gradient(gpu_lib, H, W):
    from paper_1901_06110_gb300 import dsgnlm as D
    x = synthetic.ground_truth(max(H, 16), max(W, 16), 6, True, 81)[:H, :W].copy()
    noise = synthetic.gaussian_noise((H // 2, W // 2), 0.02, 81)
    y = host(D.lpnp_sr_observe(cuda(x), cuda(noise), 1.0, 4, boundary="symmetric"))
    want = ofw.sr_forward_sym(x.astype(np.float64), PSF) + noise.astype(np.float64)
    np.testing.assert_allclose(y, want, atol=1e-6)
    den = D.dsgnlm_create()
    xv = np.random.default_rng(3).uniform(0, 1, (H, W)).astype(np.float32)
    p = D.Problem("sr", den, cuda(xv), cuda(xv), cuda(xv), alpha=1.0, y=cuda(want.astype(np.float32)),
                  boundary="symmetric")
    g = host(D.lpnp_gradient(p, cuda(xv)))
    gw = ofw.sr_grad_sym(xv.astype(np.float64), want.astype(np.float32).astype(np.float64), PSF)
    np.testing.assert_allclose(g, gw, atol=2e-6)


def test_symmetric_blur_needs_room(gpu_lib):
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    with pytest.raises(D.DsgnlmError) as e:
        D.lpnp_sr_observe(cuda(np.zeros((6, 8), np.float32)), None, 1.0, 4, boundary="symmetric")
    assert e.value.status == _abi.EINVAL


def _solver(wl, H, W):
    from paper_1901_06110_gb300 import pipeline
    return pipeline.Solver(H, W, pipeline.Params.from_workload(wl, boundary="symmetric"))


@pytest.mark.parametrize("H,W,iters", [(48, 64, 10), (30, 52, 6)])
def test_linearized_symmetric_solve_matches_oracle(gpu_lib, H, W, iters):
    wl = dict(synthetic.workload("sr64"), search_r=5, tol=1e-6, iters=iters)
    inst = problems.sr_instance_sym(wl, H=H, W=W)
    ref = problems.solve_sr_sym(wl, inst)
    s = _solver(wl, H, W)
    hist = s.run(cuda(inst["y"]), residuals=True)
    torch.cuda.synchronize()
    assert rel_l2(host(s.x), ref["x"]) <= 1e-5
    assert rel_l2(host(s.v), ref["v"]) <= 1e-5
    for (p, d), (po, do, _) in zip(hist, ref["hist"]):
        assert abs(p - po) <= 1e-6 + 1e-3 * po
    s.close()


@pytest.mark.parametrize("H,W,iters,cg", [(48, 64, 6, 5), (32, 40, 4, 12)])
def test_standard_admm_matches_oracle(gpu_lib, H, W, iters, cg):
    wl = dict(synthetic.workload("sr64"), search_r=5, tol=1e-6, iters=iters)
    inst = problems.sr_instance_sym(wl, H=H, W=W)
    ref = problems.solve_sr_sym(wl, inst, standard_cg_iters=cg)
    s = _solver(wl, H, W)
    s.prepare(cuda(inst["y"]))
    hist = s.run_standard(cuda(inst["y"]), cg, residuals=True)
    torch.cuda.synchronize()
    assert rel_l2(host(s.x), ref["x"]) <= 1e-5
    assert rel_l2(host(s.v), ref["v"]) <= 1e-5
    np.testing.assert_allclose(host(s.u), ref["u"], atol=2e-5)
    for (p, d), (po, do, _) in zip(hist, ref["hist"]):
        assert abs(p - po) <= 1e-6 + 1e-3 * po
        assert abs(d - do) <= 1e-6 + 1e-3 * do
    s.close()


def test_standard_admm_argument_checks(gpu_lib):
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    wl = dict(synthetic.workload("sr64"), search_r=5, iters=2)
    inst = problems.sr_instance_sym(wl, H=32, W=32)
    s = _solver(wl, 32, 32)
    s.prepare(cuda(inst["y"]))
    with pytest.raises(D.DsgnlmError) as e:
        s.run_standard(cuda(inst["y"]), 0)
    assert e.value.status == _abi.EINVAL
    counts = cuda(np.zeros((32, 32), np.uint8))
    p = D.Problem("spi", s.den, s.x, s.v, s.u, alpha=64.0, counts=counts)
    with pytest.raises(D.DsgnlmError) as e:
        D.lpnp_solve_standard(p, 1.0, 2, 3)
    assert e.value.status == _abi.EINVAL
    s.close()
