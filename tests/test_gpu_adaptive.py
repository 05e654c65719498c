"""Algorithm 1 with W rebuilt from the denoiser input x + u (Sec. 4: A-DSG-NLM, and
the adapt-then-freeze F-DSG-NLM schedule) through lpnp_solve_adaptive, against the
FP64 oracle.  Every adaptation balances to tol 1e-6 on both sides, so the weights
differ by at most that much; iterates are compared at 1e-5 relative."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import problems
from tests.gpu_helpers import cuda, host, rel_l2

pytestmark = pytest.mark.gpu


def _sr_case(H, W, rs):
    wl = dict(synthetic.workload("sr64"), search_r=rs, tol=1e-6)
    return wl, problems.sr_instance(wl, H=H, W=W)


@pytest.mark.parametrize("H,W,rs,iters,adapt", [(48, 64, 5, 8, 8), (48, 64, 5, 12, 4), (30, 132, 3, 5, 2)])
def test_sr_adaptive_matches_oracle(gpu_lib, H, W, rs, iters, adapt):
    from paper_1901_06110_gb300 import dsgnlm as D
    from paper_1901_06110_gb300 import pipeline
    wl, inst = _sr_case(H, W, rs)
    ref = problems.solve_sr_adaptive(wl, inst, adapt, iters=iters)
    s = pipeline.Solver(H, W, pipeline.Params.from_workload(wl, iters=iters))
    hist = s.run_adaptive(cuda(inst["y"]), adapt, residuals=True)
    torch.cuda.synchronize()
    assert rel_l2(host(s.x), ref["x"]) <= 1e-5
    assert rel_l2(host(s.v), ref["v"]) <= 1e-5
    np.testing.assert_allclose(host(s.u), ref["u"], atol=2e-5)
    for (p, d), (po, do, _) in zip(hist, ref["hist"]):
        assert abs(p - po) <= 1e-6 + 1e-3 * po
        assert abs(d - do) <= 1e-6 + 1e-3 * do
    # the handle holds the last W
    z = np.random.default_rng(2).uniform(0, 1, (H, W)).astype(np.float32)
    got = host(D.dsgnlm_apply(s.den, cuda(z)))
    want = (ref["W_last"] @ z.astype(np.float64).ravel()).reshape(H, W)
    assert rel_l2(got, want) <= 1e-5
    s.close()


def test_spi_adaptive_matches_oracle(gpu_lib):
    from paper_1901_06110_gb300 import dsgnlm as D
    from paper_1901_06110_gb300 import pipeline
    wl = dict(synthetic.workload("spi512"), search_r=4, patch_r=2, tol=1e-6)
    inst = problems.spi_instance(wl, H=40, W=56)
    ref = problems.solve_spi_adaptive(wl, inst, 3, iters=6)
    s = pipeline.Solver(40, 56, pipeline.Params.from_workload(wl, iters=6), kind="spi")
    s.run_adaptive(cuda(inst["counts"].astype(np.uint8)), 3)
    torch.cuda.synchronize()
    assert rel_l2(host(s.x), ref["x"]) <= 1e-5
    assert rel_l2(host(s.v), ref["v"]) <= 1e-5
    s.close()


def test_adaptive_argument_checks(gpu_lib):
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    wl, inst = _sr_case(16, 16, 2)
    den = D.dsgnlm_create()
    x = cuda(np.full((16, 16), 0.5, np.float32))
    v, u = x.clone(), torch.zeros_like(x)
    p = D.Problem("sr", den, x, v, u, alpha=1.0, y=cuda(inst["y"]))
    for args in [(3, 0, 2, 2), (3, 1, 2, 9), (3, 1, -1, 2)]:
        iters, adapt, rp, rs = args
        with pytest.raises(D.DsgnlmError) as e:
            D.lpnp_solve_adaptive(p, 1.0, iters, adapt, rp, rs, 0.1, 1e-6, 100)
        assert e.value.status == _abi.EINVAL
    D.lpnp_solve_adaptive(p, 1.0, 3, 1, 1, 2, 0.1, 1e-6, 100)  # den need not be built beforehand
