"""Batched Algorithm 1 (many uneven images, one launch per step) through the C ABI.

- The batched solve runs the same kernels on the same tiles as lpnp_solve, so its
  results must be bit-identical to solving the images one by one.
- Low-precision weights (FP16, BF16; FP32 arithmetic) must give the PSNR of the
  plain FP32 form within 0.01 dB, and stay close to the FP64 oracle.
"""
import numpy as np
import pytest
import torch

import synthetic
from oracle import lpnp as olp
from oracle import problems
from tests.gpu_helpers import cuda, host, rel_l2

pytestmark = pytest.mark.gpu

SIZES = [(48, 64), (96, 160), (40, 72), (130, 136)]


def _prepare(wl, H, W, seed, dtype="f32", kind="sr"):
    from paper_1901_06110_gb300 import dsgnlm as D
    if kind == "sr":
        inst = problems.sr_instance(wl, H=H, W=W, seed=seed)
        data = cuda(inst["y"])
        guide = D.lpnp_sr_guide(data)
    else:
        inst = problems.spi_instance(wl, H=H, W=W, seed=seed)
        data = cuda(inst["counts"].astype(np.uint8))
        guide = D.lpnp_spi_guide(data, 16, wl["eta"])
    den = D.dsgnlm_create(dtype)
    D.dsgnlm_build(den, guide, wl["patch_r"], wl["search_r"], wl["h"])
    D.dsgnlm_balance(den, 1e-6, 1000)
    x, v, u = D.lpnp_init(guide)
    return dict(inst=inst, data=data, guide=guide, den=den, x=x, v=v, u=u)


def _problem(wl, st, kind="sr", x=None, v=None, u=None):
    from paper_1901_06110_gb300 import dsgnlm as D
    x = st["x"] if x is None else x
    v = st["v"] if v is None else v
    u = st["u"] if u is None else u
    if kind == "sr":
        return D.Problem("sr", st["den"], x, v, u, alpha=wl["alpha"], y=st["data"],
                         blur_sigma=wl["blur_sigma"], blur_r=wl["blur_r"])
    return D.Problem("spi", st["den"], x, v, u, alpha=wl["alpha"], counts=st["data"], K=16, eta=wl["eta"],
                     spi_eps=wl["spi_eps"])


@pytest.mark.parametrize("kind,iters", [("sr", 7), ("sr", 6), ("spi", 5)])
def test_batched_equals_one_by_one(gpu_lib, kind, iters):
    from paper_1901_06110_gb300 import dsgnlm as D
    wl = synthetic.workload("sr64" if kind == "sr" else "spi512")
    wl["search_r"] = 5
    states = [_prepare(wl, H, W, 300 + i, kind=kind) for i, (H, W) in enumerate(SIZES)]
    singles, batch = [], []
    for st in states:
        a = [t.clone() for t in (st["x"], st["v"], st["u"])]
        b = [t.clone() for t in (st["x"], st["v"], st["u"])]
        singles.append(a)
        batch.append(b)
    hs = [D.lpnp_solve(_problem(wl, st, kind, *a), wl["rho"], iters, residuals=True)
          for st, a in zip(states, singles)]
    hb = D.lpnp_solve_batched([_problem(wl, st, kind, *b) for st, b in zip(states, batch)], wl["rho"], iters,
                              residuals=True)
    torch.cuda.synchronize()
    for a, b in zip(singles, batch):
        for ta, tb in zip(a, b):
            np.testing.assert_array_equal(host(ta), host(tb))
    for ha, hb_ in zip(hs, hb):
        np.testing.assert_allclose(np.array(ha), np.array(hb_), rtol=0, atol=0)


@pytest.mark.parametrize("dtype,oracle_tol", [("f16", 2e-3), ("bf16", 1.5e-2)])
def test_low_precision_batch_psnr(gpu_lib, dtype, oracle_tol):
    from paper_1901_06110_gb300 import dsgnlm as D
    wl = synthetic.workload("sr512")
    wl["search_r"] = 7
    wl["patch_r"] = 2
    sizes = [(96, 96), (128, 64), (64, 160)]
    iters = 12
    res = {}
    for dt in ("f32", dtype):
        states = [_prepare(wl, H, W, 700 + i, dtype=dt) for i, (H, W) in enumerate(sizes)]
        D.lpnp_solve_batched([_problem(wl, st) for st in states], wl["rho"], iters)
        torch.cuda.synchronize()
        res[dt] = [(host(st["x"]), st["inst"]) for st in states]
    for (x32, inst), (xlp, _) in zip(res["f32"], res[dtype]):
        truth = inst["x_true"]
        dpsnr = abs(olp.psnr(xlp, truth) - olp.psnr(x32, truth))
        assert dpsnr <= 0.01, dpsnr
        ref = problems.solve_sr(wl, inst, iters=iters, tol=1e-6)
        assert rel_l2(x32, ref["x"]) <= 1e-5
        assert rel_l2(xlp, ref["x"]) <= oracle_tol


def test_batched_rejects_mixed(gpu_lib):
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    wl = synthetic.workload("sr64")
    a = _prepare(wl, 32, 32, 1, dtype="f32")
    b = _prepare(wl, 32, 48, 2, dtype="f16")
    with pytest.raises(D.DsgnlmError) as e:
        D.lpnp_solve_batched([_problem(wl, a), _problem(wl, b)], 1.0, 2)
    assert e.value.status == _abi.EINVAL
    with pytest.raises(D.DsgnlmError) as e:  # the same handle twice
        D.lpnp_solve_batched([_problem(wl, a), _problem(wl, a)], 1.0, 2)
    assert e.value.status == _abi.EINVAL


def test_batched_schedules_agree_and_replay(gpu_lib):
    """Other offset schedules change only the FP32 summation order; a second call
    with the same batch replays the recorded graph and repeats the first exactly."""
    from paper_1901_06110_gb300 import dsgnlm as D
    wl = synthetic.workload("sr64")
    wl["search_r"] = 5
    states = [_prepare(wl, H, W, 400 + i) for i, (H, W) in enumerate(SIZES)]
    init = [[t.clone() for t in (st["x"], st["v"], st["u"])] for st in states]
    results = {}
    for slices in (0, 1, 3, 1):
        cur = [[t.clone() for t in a] for a in init]
        D.lpnp_solve_batched([_problem(wl, st, "sr", *c) for st, c in zip(states, cur)], wl["rho"], 6,
                             slices=slices)
        torch.cuda.synchronize()
        out = [host(c[0]) for c in cur]
        if slices in results:
            for a, b in zip(results[slices], out):
                np.testing.assert_array_equal(a, b)
        results[slices] = out
    for slices in (1, 3):
        for a, b in zip(results[0], results[slices]):
            assert rel_l2(b, a) <= 1e-6


def test_tune_batched_picks_a_candidate_and_leaves_iterates(gpu_lib):
    from paper_1901_06110_gb300 import dsgnlm as D
    wl = synthetic.workload("sr64")
    wl["search_r"] = 5
    states = [_prepare(wl, H, W, 500 + i) for i, (H, W) in enumerate(SIZES)]
    probs = [_problem(wl, st) for st in states]
    before = [[host(t) for t in (st["x"], st["v"], st["u"])] for st in states]
    best, ms = D.lpnp_tune_batched(probs, wl["rho"], (0, 1, 2), 2)
    assert best in (0, 1, 2) and all(v > 0 for v in ms.values())
    assert ms[best] == min(ms.values())
    for st, b in zip(states, before):
        for t, ref in zip((st["x"], st["v"], st["u"]), b):
            np.testing.assert_array_equal(host(t), ref)


def _balance_case(dtype, sizes, rp, rs, h, seed0):
    from paper_1901_06110_gb300 import dsgnlm as D
    singles, batch = [], []
    for i, (H, W) in enumerate(sizes):
        g = cuda(np.ascontiguousarray(synthetic.ground_truth(max(H, 8), max(W, 8), 6, True, seed0 + i)[:H, :W]))
        a = D.dsgnlm_create(dtype)
        D.dsgnlm_build(a, g, rp, rs, h)
        a.H, a.W = H, W
        singles.append((a, D.dsgnlm_balance(a, 1e-6, 300)))
        b = D.dsgnlm_create(dtype)
        D.dsgnlm_build(b, g, rp, rs, h)
        b.H, b.W = H, W
        batch.append(b)
    return singles, batch


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_batched_balance_equals_single(gpu_lib, dtype):
    """dsgnlm_balance_batched runs each image's own passes (its plan, buffers and
    stopping rule) in shared launches: scalings, m, update counts, residuals and the
    resulting W must equal dsgnlm_balance on each image bit for bit.  Uneven sizes
    give different tile counts, offset slices and pass counts."""
    from paper_1901_06110_gb300 import dsgnlm as D
    sizes = [(96, 96), (128, 64), (40, 200), (200, 136), (17, 33)]
    singles, batch = _balance_case(dtype, sizes, 2, 5, 0.1, 900)
    res = D.dsgnlm_balance_batched(batch, 1e-6, 300)
    assert len({r[1] for r in res}) > 1  # the images stop after different pass counts
    for (a, sa), b, rb in zip(singles, batch, res):
        assert rb[0] == sa[0] and rb[1] == sa[1] and rb[2] == sa[2], (rb, sa)
        da, ma = D.dsgnlm_copy_scaling(a)
        db, mb = D.dsgnlm_copy_scaling(b)
        assert ma == mb
        np.testing.assert_array_equal(host(da), host(db))
        z = cuda(np.random.default_rng(3).uniform(0, 1, (a.H, a.W)).astype(np.float32))
        np.testing.assert_array_equal(host(D.dsgnlm_apply(a, z)), host(D.dsgnlm_apply(b, z)))


def test_batched_balance_maxit_and_errors(gpu_lib):
    """maxit bounds every image (NOT_CONVERGED where tol is not reached, as the single
    call reports); a repeated handle or mismatched search radius is rejected."""
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    sizes = [(64, 64), (48, 130)]
    singles, batch = _balance_case("f32", sizes, 2, 4, 0.1, 950)
    res = D.dsgnlm_balance_batched(batch, 1e-12, 3)
    for (a, _), b, rb in zip(singles, batch, res):
        sa = D.dsgnlm_balance(a, 1e-12, 3)
        assert rb == sa and rb[0] == _abi.NOT_CONVERGED and rb[1] == 3
    with pytest.raises(D.DsgnlmError) as e:
        D.dsgnlm_balance_batched([batch[0], batch[0]], 1e-6, 10)
    assert e.value.status == _abi.EINVAL
    other = D.dsgnlm_create("f32")
    D.dsgnlm_build(other, cuda(np.ones((32, 32), np.float32)), 2, 3, 0.1)
    with pytest.raises(D.DsgnlmError) as e:
        D.dsgnlm_balance_batched([batch[0], other], 1e-6, 10)
    assert e.value.status == _abi.EINVAL


def test_batched_balance_schedule(gpu_lib):
    """Another offset schedule changes only the order of FP32 sums: every image still
    reaches tol with a doubly stochastic W, and its scaling stays within 1e-5 of the
    image's own balance."""
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    sizes = [(96, 96), (128, 64), (40, 200), (200, 136)]
    singles, batch = _balance_case("f32", sizes, 2, 5, 0.1, 970)
    res = D.dsgnlm_balance_batched(batch, 1e-6, 300, slices=1)
    for (a, sa), b, rb in zip(singles, batch, res):
        assert rb[0] == _abi.OK and rb[2] <= 1e-6 and abs(rb[1] - sa[1]) <= 1
        da, _ = D.dsgnlm_copy_scaling(a)
        db, _ = D.dsgnlm_copy_scaling(b)
        assert rel_l2(host(db), host(da)) <= 1e-5
        ones = torch.ones((b.H, b.W), device="cuda")
        np.testing.assert_allclose(host(D.dsgnlm_apply(b, ones)), 1.0, atol=1e-6)


def test_batched_balance_edges(gpu_lib):
    """A batch of one is the single call; a tolerance every image meets on its first
    pass stops every image there (no update), and W stays doubly stochastic."""
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    singles, batch = _balance_case("f32", [(72, 56)], 2, 3, 0.1, 990)
    (a, sa), b = singles[0], batch[0]
    assert D.dsgnlm_balance_batched([b], 1e-6, 300)[0] == sa
    np.testing.assert_array_equal(host(D.dsgnlm_copy_scaling(a)[0]), host(D.dsgnlm_copy_scaling(b)[0]))
    singles, batch = _balance_case("f32", [(64, 64), (40, 96), (96, 40)], 2, 3, 0.1, 995)
    res = D.dsgnlm_balance_batched(batch, 1e9, 300)
    for (a, _), b, rb in zip(singles, batch, res):
        sa = D.dsgnlm_balance(a, 1e9, 300)
        assert rb == sa and rb[0] == _abi.OK and rb[1] == 0
        ones = torch.ones((b.H, b.W), device="cuda")
        np.testing.assert_allclose(host(D.dsgnlm_apply(b, ones)), 1.0, atol=1e-6)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_batched_balance_accelerated_equals_single(gpu_lib, dtype):
    """Under the accelerated scheme each image of a batched balance takes its own
    heavy-ball passes: results equal the single-image balance bit for bit."""
    from paper_1901_06110_gb300 import dsgnlm as D
    sizes = [(96, 96), (128, 64), (40, 200), (17, 33)]
    singles, batch = [], []
    for i, (H, W) in enumerate(sizes):
        g = cuda(np.ascontiguousarray(synthetic.ground_truth(max(H, 8), max(W, 8), 6, True, 1300 + i)[:H, :W]))
        a = D.dsgnlm_create(dtype)
        D.dsgnlm_set_balance_scheme(a, "accelerated")
        D.dsgnlm_build(a, g, 2, 5, 0.1)
        a.H, a.W = H, W
        singles.append((a, D.dsgnlm_balance(a, 1e-6, 300)))
        b = D.dsgnlm_create(dtype)
        D.dsgnlm_set_balance_scheme(b, "accelerated")
        D.dsgnlm_build(b, g, 2, 5, 0.1)
        b.H, b.W = H, W
        batch.append(b)
    res = D.dsgnlm_balance_batched(batch, 1e-6, 300)
    for (a, sa), b, rb in zip(singles, batch, res):
        assert rb == sa, (rb, sa)
        np.testing.assert_array_equal(host(D.dsgnlm_copy_scaling(a)[0]), host(D.dsgnlm_copy_scaling(b)[0]))
