"""Hand-written adjoint of unrolled linearized PnP-ADMM (C ABI lpnp_unrolled_forward /
lpnp_backward) against FP64 references: torch autograd on the dense PyTorch form
(16x16 copy) and central finite differences of the NumPy oracle.  Tolerance 1e-4
relative (FP32 path against FP64)."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import adjoint, problems
from tests.gpu_helpers import cuda, host, rel_l2

pytestmark = pytest.mark.gpu


def _case(H, W, seed):
    wl = synthetic.workload("unroll8x256")
    inst = problems.sr_instance(wl, H=H, W=W, seed=seed)
    guide = np.clip(inst["x_true"] + 0.05 * np.random.default_rng(seed).standard_normal((H, W)), -0.05, 1.05)
    return wl, inst, guide.astype(np.float32)


def _gpu(inst, guide, h, rho, params):
    from paper_1901_06110_gb300.autograd import UnrolledSR
    y = cuda(inst["y"]).requires_grad_(True)
    g = cuda(guide).requires_grad_(True)
    ht = torch.tensor(h, dtype=torch.float64, requires_grad=True)
    rt = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
    x = UnrolledSR.apply(y, g, ht, rt, params)
    xt = cuda(inst["x_true"])
    loss = ((x - xt) ** 2).mean()
    loss.backward()
    return loss.item(), host(y.grad), host(g.grad), ht.grad.item(), rt.grad.item(), host(x.detach())


@pytest.mark.parametrize("H,W,rp,rs,T,N", [(16, 16, 2, 7, 4, 10), (16, 20, 1, 3, 2, 5),
                                            (16, 16, 1, 2, 0, 1),   # no balancing pass, one iteration
                                            (12, 16, 2, 3, 1, 2),   # one pass, H not a tile multiple
                                            (40, 72, 3, 5, 2, 3),   # 3 x 3 tiles of the extended grid
                                            (24, 40, 4, 3, 1, 2)])  # patch radius 4: D-hat planes, then box and gather
def test_adjoint_matches_torch_autograd(gpu_lib, H, W, rp, rs, T, N):
    from paper_1901_06110_gb300.autograd import UnrollParams
    wl, inst, guide = _case(H, W, 9)
    h, rho = 0.1, 1.0
    params = UnrollParams(patch_r=rp, search_r=rs, balance_passes=T, iters=N)
    loss, gy, gg, gh, gr, x = _gpu(inst, guide, h, rho, params)
    y = torch.tensor(inst["y"].astype(np.float64), requires_grad=True)
    g = torch.tensor(guide.astype(np.float64), requires_grad=True)
    ht = torch.tensor(h, dtype=torch.float64, requires_grad=True)
    rt = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
    ref = adjoint.torch_unrolled_loss(y, g, ht, rt, inst["x_true"], rp, rs, T, N)
    ref.backward()
    assert abs(loss - ref.item()) <= 1e-5 * ref.item()
    assert rel_l2(gy, y.grad.numpy()) <= 1e-4
    assert rel_l2(gg, g.grad.numpy()) <= 1e-4
    # with one iteration x_1 does not depend on W, so torch leaves h without a gradient
    href = ht.grad.item() if ht.grad is not None else 0.0
    rref = rt.grad.item() if rt.grad is not None else 0.0
    assert abs(gh - href) <= 1e-4 * abs(href) + 1e-9
    assert abs(gr - rref) <= 1e-4 * abs(rref) + 1e-9


# Finite differences.  The central difference of the FP64 oracle loss with step
# EPS has truncation error EPS^2/6 |f'''| and rounding error about u64 |f| / EPS
# (u64 = 1.1e-16, |f| ~ 2e-2): at EPS = 1e-5 that is about 1e-12 on components of
# order 1e-4 (measured against FP64 autograd: below 1e-12).  FD_FLOOR bounds it.
# The CUDA adjoint runs in FP32 (unit roundoff u32 = 2^-24 = 6e-8): a component
# near zero carries the rounding of the terms it was summed from, which are of the
# order of the largest component, so the bound adds 16 u32 max|g| (1e-6 of the
# largest component).  Every component must then match to 1e-4 of its own size:
#     |fd - g| <= 1e-4 |fd| + FD_FLOOR + 16 u32 max|g|.
EPS = 1e-5
FD_FLOOR = 1e-11
U32 = 2.0 ** -24


def _fd_points(shape, n, seed):
    rng = np.random.default_rng(seed)
    H, W = shape
    pts = [(0, 0), (H - 1, W - 1), (0, W - 1), (H // 2, W // 2)]
    while len(pts) < n:
        p = (int(rng.integers(0, H)), int(rng.integers(0, W)))
        if p not in pts:
            pts.append(p)
    return pts


@pytest.mark.parametrize("H,W,rp,rs,T,N", [(16, 16, 2, 7, 4, 10),   # the differentiable workload's radii
                                            (32, 48, 2, 5, 3, 6)])
def test_adjoint_matches_finite_differences(gpu_lib, H, W, rp, rs, T, N):
    from paper_1901_06110_gb300.autograd import UnrollParams
    wl, inst, guide = _case(H, W, 13)
    h, rho = 0.1, 1.0
    params = UnrollParams(patch_r=rp, search_r=rs, balance_passes=T, iters=N)
    loss, gy, gg, gh, gr, x = _gpu(inst, guide, h, rho, params)
    xt = inst["x_true"]
    g64 = guide.astype(np.float64)

    def f(yy=inst["y"], gu=g64, hh=h, rr=rho, trace=None):
        return adjoint.unrolled_loss(yy, gu, hh, rr, xt, rp, rs, T, N, trace=trace)

    base = {}
    f0 = f(trace=base)
    assert abs(loss - f0) <= 1e-5 * f0

    def check(name, grad, arr, kw, points):
        floor = FD_FLOOR + 16 * U32 * np.abs(grad).max()
        checked = 0
        for idx in points:
            tp, tm = {}, {}
            ap = np.array(arr, dtype=np.float64, copy=True)
            am = np.array(arr, dtype=np.float64, copy=True)
            ap[idx] += EPS
            am[idx] -= EPS
            fp = f(**{kw: ap}, trace=tp)
            fm = f(**{kw: am}, trace=tm)
            if not (adjoint.same_branches(tp, base) and adjoint.same_branches(tm, base)):
                continue  # the step crosses a kink of Pi_C or of m (reading of the differentiable form)
            fd = (fp - fm) / (2 * EPS)
            assert abs(fd - grad[idx]) <= 1e-4 * abs(fd) + floor, (name, idx, fd, grad[idx], floor)
            checked += 1
        assert checked >= 10, (name, checked)

    check("y", gy, inst["y"], "yy", _fd_points(inst["y"].shape, 12, 1))
    check("guide", gg, g64, "gu", _fd_points(g64.shape, 12, 2))
    for name, grad, val, kw in (("h", gh, h, "hh"), ("rho", gr, rho, "rr")):
        tp, tm = {}, {}
        fp = f(**{kw: val + EPS}, trace=tp)
        fm = f(**{kw: val - EPS}, trace=tm)
        assert adjoint.same_branches(tp, base) and adjoint.same_branches(tm, base), name
        fd = (fp - fm) / (2 * EPS)
        assert abs(fd - grad) <= 1e-4 * abs(fd) + FD_FLOOR, (name, fd, grad)


def _explicit(fn, y, g, h, rho, xbar):
    """x_N and the cotangents for the given cotangent of x_N."""
    y = y.clone().requires_grad_(True)
    g = g.clone().requires_grad_(True)
    ht = torch.tensor(h, dtype=torch.float64, requires_grad=True)
    rt = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
    x = fn(y, g, ht, rt)
    x.backward(xbar)
    return host(x.detach()), host(y.grad), host(g.grad), ht.grad.item(), rt.grad.item()


def test_batched_matches_single_bit_for_bit(gpu_lib):
    """The batched calls (one stream per image) give every image's x_N and
    cotangents exactly as the single-image calls where the offset split is the same
    (at 32x48 every column offset is its own slice for one image and for three); the
    scalar cotangents are the sums of the per-image values.  Repeated calls reuse the
    pooled slots."""
    from paper_1901_06110_gb300.autograd import UnrollParams, UnrolledSR, unrolled_sr
    H, W, B = 32, 48, 3
    params = UnrollParams(patch_r=2, search_r=5, balance_passes=3, iters=6)
    cases = [_case(H, W, 20 + b) for b in range(B)]
    ys = [cuda(inst["y"]) for _, inst, _ in cases]
    gs = [cuda(guide) for _, _, guide in cases]
    xbars = [cuda(np.random.default_rng(30 + b).standard_normal((H, W)).astype(np.float32)) for b in range(B)]
    h, rho = 0.1, 1.0
    single = lambda y, g, ht, rt: UnrolledSR.apply(y, g, ht, rt, params)
    singles = [_explicit(single, ys[b], gs[b], h, rho, xbars[b]) for b in range(B)]
    batched = lambda y, g, ht, rt: unrolled_sr(y, g, ht, rt, params)
    for _ in range(2):
        xb, gyb, ggb, hb, rb = _explicit(batched, torch.stack(ys), torch.stack(gs), h, rho, torch.stack(xbars))
        for b in range(B):
            assert np.array_equal(xb[b], singles[b][0])
            assert np.array_equal(gyb[b], singles[b][1])
            assert np.array_equal(ggb[b], singles[b][2])
        assert hb == sum(s[3] for s in singles)
        assert rb == sum(s[4] for s in singles)
    again = _explicit(single, ys[1], gs[1], h, rho, xbars[1])
    for a, b_ in zip(again, singles[1]):
        assert np.array_equal(a, b_)


def test_batched_split_for_the_batch(gpu_lib):
    """At 256^2 the batch of four sizes each handle's offset split for four images at
    once (fewer slices than one image alone), so W's partial sums are added in another
    order: the results agree with the single-image calls to FP32 rounding and are
    bitwise repeatable."""
    from paper_1901_06110_gb300.autograd import UnrollParams, UnrolledSR, unrolled_sr
    H, W, B = 256, 256, 4
    params = UnrollParams(patch_r=2, search_r=7, balance_passes=4, iters=10)
    cases = [_case(H, W, 40 + b) for b in range(B)]
    ys = [cuda(inst["y"]) for _, inst, _ in cases]
    gs = [cuda(guide) for _, _, guide in cases]
    xbars = [cuda(np.random.default_rng(50 + b).standard_normal((H, W)).astype(np.float32)) for b in range(B)]
    h, rho = 0.1, 1.0
    single = lambda y, g, ht, rt: UnrolledSR.apply(y, g, ht, rt, params)
    singles = [_explicit(single, ys[b], gs[b], h, rho, xbars[b]) for b in range(B)]
    batched = lambda y, g, ht, rt: unrolled_sr(y, g, ht, rt, params)
    runs = [_explicit(batched, torch.stack(ys), torch.stack(gs), h, rho, torch.stack(xbars)) for _ in range(2)]
    for a, b_ in zip(runs[0], runs[1]):
        assert np.array_equal(a, b_)
    xb, gyb, ggb, hb, rb = runs[0]
    for b in range(B):
        assert rel_l2(xb[b], singles[b][0]) <= 1e-5
        assert rel_l2(gyb[b], singles[b][1]) <= 1e-5
        assert rel_l2(ggb[b], singles[b][2]) <= 1e-5
    hs = sum(s[3] for s in singles)
    rs_ = sum(s[4] for s in singles)
    assert abs(hb - hs) <= 1e-5 * abs(hs)
    assert abs(rb - rs_) <= 1e-5 * abs(rs_)


def test_batched_repeated_calls_follow_new_inputs(gpu_lib):
    """Repeated batched calls on pooled tapes and handles, with new inputs every call:
    each gives the single-image results on its own inputs bit for bit, and launches
    the same number of kernels."""
    from paper_1901_06110_gb300 import dsgnlm as D
    from paper_1901_06110_gb300.autograd import UnrollParams, UnrolledSR, unrolled_sr
    H, W, B = 32, 48, 3
    params = UnrollParams(patch_r=2, search_r=5, balance_passes=3, iters=6)
    single = lambda y, g, ht, rt: UnrolledSR.apply(y, g, ht, rt, params)
    batched = lambda y, g, ht, rt: unrolled_sr(y, g, ht, rt, params)
    h, rho = 0.1, 1.0
    launches = []
    for call in range(5):
        cases = [_case(H, W, 60 + 7 * call + b) for b in range(B)]
        ys = [cuda(inst["y"]) for _, inst, _ in cases]
        gs = [cuda(guide) for _, _, guide in cases]
        xbars = [cuda(np.random.default_rng(80 + call + b).standard_normal((H, W)).astype(np.float32))
                 for b in range(B)]
        n0 = D.dsgnlm_launch_count()
        xb, gyb, ggb, hb, rb = _explicit(batched, torch.stack(ys), torch.stack(gs), h, rho, torch.stack(xbars))
        launches.append(D.dsgnlm_launch_count() - n0)
        singles = [_explicit(single, ys[b], gs[b], h, rho, xbars[b]) for b in range(B)]
        for b in range(B):
            assert np.array_equal(xb[b], singles[b][0]), (call, b)
            assert np.array_equal(gyb[b], singles[b][1]), (call, b)
            assert np.array_equal(ggb[b], singles[b][2]), (call, b)
        assert hb == sum(s[3] for s in singles)
        assert rb == sum(s[4] for s in singles)
    assert len(set(launches)) == 1, launches


def test_handle_after_unrolled_forward_applies_its_w(gpu_lib):
    """The unrolled forward leaves its W on the handle, with m and 1/m formed on the
    device; a later host-side call on the handle (apply, copy of the scaling) reads
    them back and applies the W of Eqs. S1-S3 after exactly T balancing passes."""
    from oracle import dsgnlm as odsg
    from paper_1901_06110_gb300 import dsgnlm as D
    from paper_1901_06110_gb300.autograd import UnrollParams, UnrolledSR
    H, W, rp, rs, T, N = 24, 32, 2, 3, 2, 2
    wl, inst, guide = _case(H, W, 17)
    params = UnrollParams(patch_r=rp, search_r=rs, balance_passes=T, iters=N)
    slot_x = UnrolledSR.apply(cuda(inst["y"]), cuda(guide), 0.1, 1.0, params)
    torch.cuda.synchronize()
    from paper_1901_06110_gb300 import autograd as A
    lib = A._abi.load()
    tp = A._Slot()
    x_out = torch.empty((H, W), device="cuda")
    y = cuda(inst["y"])
    g = cuda(guide)
    D._check(lib.lpnp_unrolled_forward(tp.ptr, tp.den.handle, y.data_ptr(), g.data_ptr(), H, W, rp, rs, 0.1, T, 1.0,
                                       1.0, N, 1.0, 4, x_out.data_ptr()), "lpnp_unrolled_forward")
    tp.den.H, tp.den.W = H, W
    K1 = odsg.kernel_matrix(guide.astype(np.float64), rp, rs, 0.1)
    d_o, _, _ = odsg.sinkhorn(K1, 0.0, T)
    W_o, m_o = odsg.dsg_matrix(K1, d_o)
    d, m = D.dsgnlm_copy_scaling(tp.den)
    assert abs(m - m_o) <= 1e-5 * m_o
    np.testing.assert_allclose(host(d).ravel(), d_o, rtol=1e-5)
    z = np.random.default_rng(5).uniform(0, 1, (H, W)).astype(np.float32)
    out = host(D.dsgnlm_apply(tp.den, cuda(z)))
    assert rel_l2(out, odsg.denoise(W_o, z.astype(np.float64))) <= 1e-5
    np.testing.assert_array_equal(host(x_out), host(slot_x))
