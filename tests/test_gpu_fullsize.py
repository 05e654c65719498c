"""Parity at the full 512x512 super-resolution workload (7x7 patches, 21x21 window,
h = 0.08, balance to 1e-6, 30 iterations), in the launch configuration the
benchmark times (the same pipeline calls).  Weights, balance and apply are
checked at sampled pixels against oracle rows computed one by one, the balance
and the denoiser through properties that hold at any size, and the final iterate
against the full FP64 oracle solve."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import dsgnlm as odsg
from oracle import problems
from tests.gpu_helpers import cuda, half_offsets, host, rel_l2

pytestmark = pytest.mark.gpu

WL = synthetic.workload("sr512")


@pytest.fixture(scope="module")
def solved(gpu_lib):
    from paper_1901_06110_gb300 import pipeline
    inst = problems.sr_instance(WL)
    params = pipeline.Params.from_workload(WL)
    solver = pipeline.Solver(WL["H"], WL["W"], params)
    hist = solver.run(cuda(inst["y"]), residuals=True)
    torch.cuda.synchronize()
    return dict(inst=inst, solver=solver, hist=hist)


def _samples(H, W, n=40, seed=0):
    rng = np.random.default_rng(seed)
    pts = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (H // 2, 3), (5, W // 2)]
    pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, H, n), rng.integers(0, W, n))]
    return pts


def test_weights_at_sampled_pixels(solved):
    from paper_1901_06110_gb300 import dsgnlm as D
    s = solved["solver"]
    guide = host(s.guide)
    planes = D.dsgnlm_copy_weights(s.den)
    rs = WL["search_r"]
    offs = half_offsets(rs)
    for (i, j) in _samples(512, 512):
        row = odsg.kernel_row(guide, WL["patch_r"], rs, WL["h"], (i, j))
        got = host(planes[:, i, j])
        for k, (oy, ox) in enumerate(offs):
            want = row.get((i + oy, j + ox), 0.0)
            assert abs(got[k] - want) <= 1e-5 * want + 2e-7, (i, j, oy, ox)


def test_balance_and_apply_at_sampled_pixels(solved):
    from paper_1901_06110_gb300 import dsgnlm as D
    s = solved["solver"]
    st, k, res = s.balance
    assert st == 0 and res <= WL["tol"]
    guide = host(s.guide)
    d_t, m = D.dsgnlm_copy_scaling(s.den)
    d = host(d_t)
    z = np.random.default_rng(1).uniform(0, 1, (512, 512)).astype(np.float32)
    y = host(D.dsgnlm_apply(s.den, cuda(z)))
    for (i, j) in _samples(512, 512, 24, 2):
        row = odsg.kernel_row(guide, WL["patch_r"], WL["search_r"], WL["h"], (i, j))
        # row sum of diag(d) K1 diag(d) with the oracle kernel: balanced to tol
        rsum = d[i, j] * sum(val * d[r] for r, val in row.items())
        assert abs(rsum - 1.0) <= 5 * WL["tol"]
        # y_s = sum_{r != s} W_sr z_r + (1 - sum_{r != s} W_sr) z_s, W_sr = d_s d_r K1 / m
        off = {r: d[i, j] * d[r] * val / m for r, val in row.items() if r != (i, j)}
        want = sum(w * z[r] for r, w in off.items()) + (1.0 - sum(off.values())) * z[i, j]
        assert abs(y[i, j] - want) <= 1e-5 * abs(want) + 1e-6


def test_denoiser_properties_full_size(solved):
    from paper_1901_06110_gb300 import dsgnlm as D
    s = solved["solver"]
    ones = torch.ones((512, 512), device="cuda")
    np.testing.assert_allclose(host(D.dsgnlm_apply(s.den, ones)), 1.0, atol=1e-6)
    z = torch.rand((512, 512), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    y = D.dsgnlm_apply(s.den, z)
    assert abs(float(y.double().sum()) - float(z.double().sum())) <= 1e-5 * float(z.double().sum())
    # symmetry: <W a, b> = <a, W b>
    a = torch.rand((512, 512), device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    lhs = float((D.dsgnlm_apply(s.den, a).double() * z.double()).sum())
    rhs = float((a.double() * y.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_full_solve_matches_oracle(solved):
    ref = problems.solve_sr(WL, solved["inst"], tol=WL["tol"])
    s = solved["solver"]
    assert rel_l2(host(s.x), ref["x"]) <= 1e-5
    assert rel_l2(host(s.v), ref["v"]) <= 1e-5
    np.testing.assert_allclose(host(s.x), ref["x"], atol=5e-5)
    p_gpu, d_gpu = solved["hist"][-1]
    p_o, d_o, _ = ref["hist"][-1]
    assert abs(p_gpu - p_o) <= 1e-6 + 1e-2 * p_o
    assert abs(d_gpu - d_o) <= 1e-6 + 1e-2 * d_o
