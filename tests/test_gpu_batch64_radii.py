"""Batched Algorithm 1 at the radii and parameters of the 64-image workload (7x7
patches, 21x21 window, h = 0.08, balance to 1e-6, 30 iterations), in the launch
configuration the benchmark times (`pipeline.BatchSolver`: batched balance, then
one launch per step over every image's tiles, replayed from a CUDA graph).

Images of uneven sizes: 512^2, a ragged 136x200 (neither side a multiple of the
16x128 stencil tile), 256^2 and 128^2, seeds 1004 + i as in the workload recipe.
Every weight storage type (FP32, FP16, BF16) runs under each handle's own offset
plan (slices = 0) and under the one-slice schedule the autotuner picks for the
64-image batch (slices = 1).

Checked against the FP64 oracle (method of Sec. 3, Eqs. NLM, S1-S3, inside
Algorithm 1):
- every image's x and v against the full oracle solve: FP32 within 1e-5 relative,
  FP16 within 2e-3, BF16 within 1.5e-2 (a stored FP16/BF16 weight carries a
  relative rounding error up to 2^-11 / 2^-8);
- every image's PSNR within 0.01 dB of the plain FP32 form solved one image at a
  time (`pipeline.Solver`);
- on the 512^2 image, the stored weights at sampled pixels against oracle kernel
  rows (FP32 to 1e-5 relative; FP16/BF16 to half a unit in the last place of the
  storage type on top of that), the balanced row sums and W z at sampled pixels
  (FP32), and W 1 = 1, sum preservation and <W a, b> = <a, W b> (every type).
"""
import numpy as np
import pytest
import torch

import synthetic
from oracle import dsgnlm as odsg
from oracle import lpnp as olp
from oracle import problems
from tests.gpu_helpers import cuda, half_offsets, host, rel_l2

pytestmark = pytest.mark.gpu

WL = synthetic.workload("batch64")
SIZES = [(512, 512), (136, 200), (256, 256), (128, 128)]
ORACLE_TOL = {"f32": 1e-5, "f16": 2e-3, "bf16": 1.5e-2}
# half a unit in the last place of the storage type, relative (round to nearest)
HALF_ULP = {"f32": 0.0, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}
# absolute floor: FP16 spacing below its smallest normal (2^-24) halved; FP32 weights
# that underflow in the exponential
ABS_FLOOR = {"f32": 2e-7, "f16": 2e-7 + 2.0 ** -25, "bf16": 2e-7}


@pytest.fixture(scope="module")
def instances():
    """Instances and the FP64 oracle solves (kept: x, v, history; the matrices are
    dropped to bound host memory)."""
    out = []
    for i, (H, W) in enumerate(SIZES):
        inst = problems.sr_instance(WL, H=H, W=W, seed=WL["seed"] + i)
        ref = problems.solve_sr(WL, inst, iters=WL["iters"], tol=WL["tol"])
        out.append(dict(inst=inst, x=ref["x"], v=ref["v"], hist=ref["hist"], updates=ref["info"]["updates"]))
        del ref
    return out


@pytest.fixture(scope="module")
def plain_fp32(gpu_lib, instances):
    """The plain FP32 form: each image solved alone (pipeline.Solver)."""
    from paper_1901_06110_gb300 import pipeline
    params = pipeline.Params.from_workload(WL)
    res = []
    for (H, W), it in zip(SIZES, instances):
        s = pipeline.Solver(H, W, params)
        s.run(cuda(it["inst"]["y"]))
        torch.cuda.synchronize()
        res.append(dict(x=host(s.x), v=host(s.v), balance=s.balance))
        s.close()
    return res


@pytest.fixture(scope="module", params=[("f32", 0), ("f32", 1), ("f16", 0), ("f16", 1), ("bf16", 0), ("bf16", 1)],
                ids=lambda p: f"{p[0]}-slices{p[1]}")
def batched(request, gpu_lib, instances):
    from paper_1901_06110_gb300 import pipeline
    dtype, slices = request.param
    params = pipeline.Params.from_workload(WL, weight_dtype=dtype)
    bs = pipeline.BatchSolver(SIZES, params)
    bs.slices = slices
    ys = [cuda(it["inst"]["y"]) for it in instances]
    hist = bs.run(ys, residuals=True)
    torch.cuda.synchronize()
    yield dict(dtype=dtype, slices=slices, bs=bs, hist=hist,
               x=[host(t) for t in bs.x], v=[host(t) for t in bs.v], guide=[host(t) for t in bs.guide])
    bs.close()


def test_batched_matches_oracle_and_plain_psnr(batched, instances, plain_fp32):
    tol = ORACLE_TOL[batched["dtype"]]
    for k, ((H, W), it, pl) in enumerate(zip(SIZES, instances, plain_fp32)):
        st, upd, res = batched["bs"].balance[k]
        assert st == 0 and res <= WL["tol"], (k, batched["bs"].balance[k])
        x, v = batched["x"][k], batched["v"][k]
        assert x.min() >= 0.0 and x.max() <= 1.0
        ex, ev = rel_l2(x, it["x"]), rel_l2(v, it["v"])
        assert ex <= tol and ev <= tol, (k, H, W, ex, ev)
        truth = it["inst"]["x_true"]
        dpsnr = abs(olp.psnr(x, truth) - olp.psnr(pl["x"], truth))
        assert dpsnr <= 0.01, (k, dpsnr)
        p_gpu, d_gpu = batched["hist"][k][-1]
        p_o, d_o, _ = it["hist"][-1]
        if batched["dtype"] == "f32":
            assert abs(p_gpu - p_o) <= 1e-6 + 1e-2 * p_o
            assert abs(d_gpu - d_o) <= 1e-6 + 1e-2 * d_o


def test_batched_f32_own_plans_equal_plain(batched, plain_fp32):
    """FP32 under each handle's own plan runs the single-image arithmetic in the same
    order (batched balance and batched steps), so it equals the plain form bit for bit."""
    if batched["dtype"] != "f32" or batched["slices"] != 0:
        pytest.skip("own plans, FP32 only")
    for k, pl in enumerate(plain_fp32):
        np.testing.assert_array_equal(batched["x"][k], pl["x"])
        np.testing.assert_array_equal(batched["v"][k], pl["v"])
        assert batched["bs"].balance[k] == pl["balance"]


def _samples(H, W, n, seed):
    rng = np.random.default_rng(seed)
    pts = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (H // 2, 3), (5, W // 2), (H - 11, W - 10)]
    pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, H, n), rng.integers(0, W, n))]
    return pts


def test_512_weights_at_sampled_pixels(batched):
    from paper_1901_06110_gb300 import dsgnlm as D
    dt = batched["dtype"]
    den = batched["bs"].dens[0]
    guide = batched["guide"][0]
    planes = D.dsgnlm_copy_weights(den).float()
    rs = WL["search_r"]
    offs = half_offsets(rs)
    H, W = SIZES[0]
    for (i, j) in _samples(H, W, 16, 11):
        row = odsg.kernel_row(guide, WL["patch_r"], rs, WL["h"], (i, j))
        got = host(planes[:, i, j])
        for k, (oy, ox) in enumerate(offs):
            want = row.get((i + oy, j + ox), 0.0)
            bound = (1e-5 + HALF_ULP[dt]) * want + ABS_FLOOR[dt]
            assert abs(got[k] - want) <= bound, (dt, i, j, oy, ox, got[k], want)


def test_512_balance_and_apply(batched):
    """Row sums of the balanced FP32 kernel and W z at sampled pixels against the
    oracle's kernel rows; for every storage type the properties of Theorem IV.1
    that survive quantisation (the closure is formed from the stored values)."""
    from paper_1901_06110_gb300 import dsgnlm as D
    den = batched["bs"].dens[0]
    H, W = SIZES[0]
    ones = torch.ones((H, W), device="cuda")
    np.testing.assert_allclose(host(D.dsgnlm_apply(den, ones)), 1.0, atol=1e-6)
    gen = torch.Generator("cuda").manual_seed(5)
    z = torch.rand((H, W), device="cuda", generator=gen)
    a = torch.rand((H, W), device="cuda", generator=gen)
    y = D.dsgnlm_apply(den, z)
    assert abs(float(y.double().sum()) - float(z.double().sum())) <= 1e-5 * float(z.double().sum())
    lhs = float((D.dsgnlm_apply(den, a).double() * z.double()).sum())
    rhs = float((a.double() * y.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    if batched["dtype"] != "f32":
        return
    guide = batched["guide"][0]
    d_t, m = D.dsgnlm_copy_scaling(den)
    d = host(d_t)
    zh, yh = host(z), host(y)
    for (i, j) in _samples(H, W, 12, 12):
        row = odsg.kernel_row(guide, WL["patch_r"], WL["search_r"], WL["h"], (i, j))
        rsum = d[i, j] * sum(val * d[r] for r, val in row.items())
        assert abs(rsum - 1.0) <= 5 * WL["tol"], (i, j, rsum)
        off = {r: d[i, j] * d[r] * val / m for r, val in row.items() if r != (i, j)}
        want = sum(w * zh[r] for r, w in off.items()) + (1.0 - sum(off.values())) * zh[i, j]
        assert abs(yh[i, j] - want) <= 1e-5 * abs(want) + 1e-6, (i, j)
