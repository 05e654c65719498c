"""GPU parity of the DSG-NLM kernels (build, balance, apply) against the FP64 oracle,
through the C ABI.  Shapes span several CUDA tiles with ragged tails, images
smaller than the search window, patch radius 0 and patch radii larger than the
image.

Tolerances (FP32 path against FP64, derived from the arithmetic): a weight
exp(-D c) carries the FP32 rounding of the patch sums (2 r_p + 1 terms per
direction) and of exp, about 1e-6 relative for weights that matter, so weights are
compared at rtol 1e-5, atol 2e-7; scalings and W z at 1e-5 relative (the north
star's FP32 target)."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import dsgnlm as odsg
from tests.gpu_helpers import cuda, half_offsets, host, planes_from_matrix, rel_l2

pytestmark = pytest.mark.gpu

CASES = [
    # H, W, patch_r, search_r, h
    (37, 45, 2, 5, 0.1),
    (40, 70, 3, 10, 0.08),
    (33, 17, 3, 4, 0.08),
    (7, 9, 1, 2, 0.3),
    (5, 6, 2, 7, 0.2),     # image smaller than the search window
    (20, 20, 0, 3, 0.1),   # 1x1 patches
    (12, 13, 10, 1, 0.5),  # patch larger than the image
    (1, 40, 1, 3, 0.2),    # single row
    (30, 35, 1, 6, 0.15),
    (24, 50, 2, 8, 0.1),
    (35, 140, 2, 12, 0.1),  # two column tiles, largest compiled radius
    (26, 29, 2, 9, 0.1),    # radius without a compiled TMA kernel: generic gather path
    (40, 300, 3, 10, 0.08),  # three column tiles, ragged, split offsets
    (30, 48, 14, 3, 0.3),    # largest patch (29 x 29): generic-radius build
    (36, 150, 5, 10, 0.1),   # Table 1 patch sizes (11, 17, 23) with the 21x21 window
    (40, 140, 8, 10, 0.1),
    (34, 136, 11, 10, 0.1),
    (48, 56, 5, 21, 0.1),    # Table 1's 43x43 reading of N_s = 21: generic gather path
]


def _guide(H, W, seed=0):
    img = synthetic.ground_truth(max(H, 8), max(W, 8), 6, True, 500 + seed)[:H, :W]
    return np.ascontiguousarray(img)


def _gpu_den(gpu_lib, guide, rp, rs, h, dtype="f32"):
    from paper_1901_06110_gb300 import dsgnlm as D
    den = D.dsgnlm_create(dtype)
    D.dsgnlm_build(den, cuda(guide), rp, rs, h)
    return den


@pytest.mark.parametrize("H,W,rp,rs,h", CASES)
def test_build_matches_oracle_kernel(gpu_lib, H, W, rp, rs, h):
    from paper_1901_06110_gb300 import dsgnlm as D
    g = _guide(H, W)
    den = _gpu_den(gpu_lib, g, rp, rs, h)
    got = host(D.dsgnlm_copy_weights(den))
    K1 = odsg.kernel_matrix(g.astype(np.float64), rp, rs, h)
    want = planes_from_matrix(K1, H, W, rs)
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=2e-7)


@pytest.mark.parametrize("H,W,rp,rs,h", CASES)
@pytest.mark.parametrize("updates", [1, 4])
def test_balance_and_apply_match_oracle(gpu_lib, H, W, rp, rs, h, updates):
    from paper_1901_06110_gb300 import dsgnlm as D
    g = _guide(H, W, 1)
    den = _gpu_den(gpu_lib, g, rp, rs, h)
    st, k, res = D.dsgnlm_balance(den, 0.0, updates)
    K1 = odsg.kernel_matrix(g.astype(np.float64), rp, rs, h)
    d_o, k_o, hist = odsg.sinkhorn(K1, 0.0, updates)
    W_o, m_o = odsg.dsg_matrix(K1, d_o)
    assert k == k_o
    d, m = D.dsgnlm_copy_scaling(den)
    np.testing.assert_allclose(host(d).ravel(), d_o, rtol=1e-5)
    assert abs(m - m_o) <= 1e-5 * m_o
    assert abs(res - hist[-1]) <= 1e-5 + 1e-4 * hist[-1]
    z = np.random.default_rng(H * W).uniform(0, 1, (H, W)).astype(np.float32)
    y = host(D.dsgnlm_apply(den, cuda(z)))
    want = odsg.denoise(W_o, z.astype(np.float64))
    assert rel_l2(y, want) <= 1e-5
    np.testing.assert_allclose(y, want, atol=1e-5)


@pytest.mark.parametrize("shape,rp,rs,h", [((6, 7), 1, 2, 0.3), ((5, 9), 2, 3, 0.15)])
def test_one_update_equals_algorithm_2(gpu_lib, shape, rp, rs, h):
    # maxit = 1 is the paper's one-shot normalisation: the CUDA path must give the
    # literal three-aggregation transcription of Algorithm 2
    from paper_1901_06110_gb300 import dsgnlm as D
    vt = np.random.default_rng(2).uniform(0, 1, shape).astype(np.float32)
    den = _gpu_den(gpu_lib, vt, rp, rs, h)
    D.dsgnlm_balance(den, 0.0, 1)
    got = host(D.dsgnlm_apply(den, cuda(vt)))
    want = odsg.alg2_literal(vt.astype(np.float64), vt.astype(np.float64), rp, rs, h)
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6)


def test_converged_balance_is_doubly_stochastic(gpu_lib):
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    H, W = 64, 48
    g = _guide(H, W, 3)
    den = _gpu_den(gpu_lib, g, 2, 5, 0.1)
    st, k, res = D.dsgnlm_balance(den, 1e-6, 1000)
    assert st == _abi.OK and res <= 1e-6
    K1 = odsg.kernel_matrix(g.astype(np.float64), 2, 5, 0.1)
    d_o, k_o, hist = odsg.sinkhorn(K1, 1e-6, 1000)
    assert abs(k - k_o) <= 1
    W_o, _ = odsg.dsg_matrix(K1, d_o)
    ones = torch.ones((H, W), device="cuda")
    np.testing.assert_allclose(host(D.dsgnlm_apply(den, ones)), 1.0, atol=1e-6)
    z = np.random.default_rng(4).uniform(0, 1, (H, W)).astype(np.float32)
    y = host(D.dsgnlm_apply(den, cuda(z)))
    assert abs(y.sum() - z.astype(np.float64).sum()) <= 1e-5 * z.sum()
    assert rel_l2(y, odsg.denoise(W_o, z.astype(np.float64))) <= 1e-5


def test_balance_statuses(gpu_lib):
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    g = _guide(40, 40, 5)
    den = _gpu_den(gpu_lib, g, 2, 5, 0.1)
    st, k, res = D.dsgnlm_balance(den, 1e-12, 2)
    assert st == _abi.NOT_CONVERGED and k == 2 and res > 1e-12
    # 1e-12 is below the FP32 floor of the scaling: the residual stalls
    st, k, res = D.dsgnlm_balance(den, 1e-12, 10000)
    assert st == _abi.STALLED and k < 10000 and res < 1e-5
    # W stays doubly stochastic whatever the stopping point
    ones = torch.ones((40, 40), device="cuda")
    np.testing.assert_allclose(host(D.dsgnlm_apply(den, ones)), 1.0, atol=1e-6)
    # maxit = 0 keeps d = 1: W = K1 / m with the closed diagonal
    st, k, res = D.dsgnlm_balance(den, 0.0, 0)
    assert st == _abi.NOT_CONVERGED and k == 0
    d, m = D.dsgnlm_copy_scaling(den)
    assert float(d.min()) == 1.0 and float(d.max()) == 1.0


def test_identity_special_cases_on_gpu(gpu_lib):
    from paper_1901_06110_gb300 import dsgnlm as D
    g = np.random.default_rng(6).uniform(0, 1, (30, 31)).astype(np.float32)
    z = np.random.default_rng(7).uniform(0, 1, (30, 31)).astype(np.float32)
    for rs, h in [(0, 0.1), (3, 1e-6)]:
        den = _gpu_den(gpu_lib, g, 1, rs, h)
        D.dsgnlm_balance(den, 1e-7, 100)
        np.testing.assert_array_equal(host(D.dsgnlm_apply(den, cuda(z))), z.astype(np.float64))


def test_low_precision_weights_stay_doubly_stochastic(gpu_lib):
    from paper_1901_06110_gb300 import dsgnlm as D
    H, W = 45, 38
    g = _guide(H, W, 8)
    z = np.random.default_rng(9).uniform(0, 1, (H, W)).astype(np.float32)
    K1 = odsg.kernel_matrix(g.astype(np.float64), 2, 4, 0.1)
    W_o, _ = odsg.build_w(g.astype(np.float64), 2, 4, 0.1, 1e-6, 1000)
    want = odsg.denoise(W_o, z.astype(np.float64))
    for dt, tdt, wtol in [("f16", torch.float16, 1e-3), ("bf16", torch.bfloat16, 8e-3)]:
        den = _gpu_den(gpu_lib, g, 2, 4, 0.1, dt)
        planes = D.dsgnlm_copy_weights(den)
        assert planes.dtype == tdt
        ref = planes_from_matrix(K1, H, W, 4)
        np.testing.assert_allclose(host(planes), ref, rtol=wtol, atol=wtol * 1e-2)
        D.dsgnlm_balance(den, 1e-6, 1000)
        ones = torch.ones((H, W), device="cuda")
        np.testing.assert_allclose(host(D.dsgnlm_apply(den, ones)), 1.0, atol=1e-6)
        y = host(D.dsgnlm_apply(den, cuda(z)))
        assert rel_l2(y, want) <= 10 * wtol


def test_deterministic(gpu_lib):
    from paper_1901_06110_gb300 import dsgnlm as D
    g = _guide(50, 60, 10)
    z = cuda(np.random.default_rng(11).uniform(0, 1, (50, 60)).astype(np.float32))
    outs = []
    for _ in range(2):
        den = _gpu_den(gpu_lib, g, 3, 6, 0.1)
        D.dsgnlm_balance(den, 1e-6, 100)
        outs.append(host(D.dsgnlm_apply(den, z)))
    np.testing.assert_array_equal(outs[0], outs[1])


def test_state_errors(gpu_lib):
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    den = D.dsgnlm_create("f32")
    x = torch.zeros((8, 8), device="cuda")
    with pytest.raises(D.DsgnlmError) as e:
        D.dsgnlm_balance(den, 1e-6, 10)
    assert e.value.status == _abi.NOT_BUILT
    D.dsgnlm_build(den, x, 1, 2, 0.1)
    den.H, den.W = 8, 8
    with pytest.raises(D.DsgnlmError) as e:
        D.dsgnlm_apply(den, x)
    assert e.value.status == _abi.NOT_BALANCED
    assert D.dsgnlm_num_offsets(den) == len(half_offsets(2))


@pytest.mark.parametrize("H,W,rp,rs,h", [(96, 80, 3, 10, 0.08), (64, 48, 2, 5, 0.1), (40, 300, 3, 10, 0.08)])
def test_accelerated_balance_reaches_the_same_w(gpu_lib, H, W, rp, rs, h):
    """The accelerated scheme (two symmetric Sinkhorn steps, then heavy-ball steps on
    log d) has the fixed point of Eq. S2 iterated, d (K1 d) = 1, which is unique: the
    scaling it reaches at tol 1e-6 is within the tolerance of the oracle's scaling
    balanced to 1e-11, in fewer passes than the plain step needs."""
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    g = _guide(H, W, 12)
    plain = _gpu_den(gpu_lib, g, rp, rs, h)
    st_p = D.dsgnlm_balance(plain, 1e-6, 1000)
    acc = _gpu_den(gpu_lib, g, rp, rs, h)
    D.dsgnlm_set_balance_scheme(acc, "accelerated")
    st_a = D.dsgnlm_balance(acc, 1e-6, 1000)
    assert st_p[0] == _abi.OK and st_a[0] == _abi.OK and st_a[2] <= 1e-6
    assert st_a[1] <= st_p[1] - 4, (st_a, st_p)
    K1 = odsg.kernel_matrix(g.astype(np.float64), rp, rs, h)
    d_o, _, hist = odsg.sinkhorn(K1, 1e-11, 10000)
    W_o, m_o = odsg.dsg_matrix(K1, d_o)
    d_a, m_a = D.dsgnlm_copy_scaling(acc)
    np.testing.assert_allclose(host(d_a).ravel(), d_o, rtol=3e-6)
    assert abs(m_a - m_o) <= 3e-6 * m_o
    ones = torch.ones((H, W), device="cuda")
    np.testing.assert_allclose(host(D.dsgnlm_apply(acc, ones)), 1.0, atol=1e-6)
    z = np.random.default_rng(13).uniform(0, 1, (H, W)).astype(np.float32)
    y = host(D.dsgnlm_apply(acc, cuda(z)))
    assert rel_l2(y, odsg.denoise(W_o, z.astype(np.float64))) <= 1e-5


@pytest.mark.parametrize("updates", [1, 2])
def test_accelerated_balance_starts_with_plain_steps(gpu_lib, updates):
    # the first two passes of the accelerated scheme are the plain step: maxit = 1
    # is still the paper's one-shot normalisation, bit for bit
    from paper_1901_06110_gb300 import dsgnlm as D
    g = _guide(48, 72, 14)
    a = _gpu_den(gpu_lib, g, 2, 5, 0.1)
    b = _gpu_den(gpu_lib, g, 2, 5, 0.1)
    D.dsgnlm_set_balance_scheme(b, "accelerated")
    assert D.dsgnlm_balance(a, 0.0, updates) == D.dsgnlm_balance(b, 0.0, updates)
    np.testing.assert_array_equal(host(D.dsgnlm_copy_scaling(a)[0]), host(D.dsgnlm_copy_scaling(b)[0]))


def test_balance_scheme_argument(gpu_lib):
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    den = D.dsgnlm_create("f32")
    assert den.lib.dsgnlm_set_balance_scheme(den.handle, 2) == _abi.EINVAL
    assert den.lib.dsgnlm_set_balance_scheme(None, 0) == _abi.EINVAL


@pytest.mark.parametrize("rp,rs", [(5, 10), (8, 10), (11, 10), (14, 10), (5, 21), (14, 21)])
def test_table1_configurations_at_256(gpu_lib, rp, rs):
    """The configurations of Table 1 (patch sizes 11-29, the 21x21 and 43x43 readings of
    N_s = 21) on a 256x256 image: stored weights at sampled pixels against oracle kernel
    rows, then the paper's one normalisation (maxit = 1, Eq. S2) with the closure of
    Eq. S3: row sums of W = 1 and W z at sampled pixels against the rows of W."""
    from paper_1901_06110_gb300 import dsgnlm as D
    g = _guide(256, 256, 20)
    h = 0.1
    den = _gpu_den(gpu_lib, g, rp, rs, h)
    planes = D.dsgnlm_copy_weights(den)
    offs = half_offsets(rs)
    rng = np.random.default_rng(rp * 100 + rs)
    pts = [(0, 0), (255, 255), (0, 255), (128, 3), (250, 128)]
    pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, 256, 7), rng.integers(0, 256, 7))]
    rows = {}
    for (i, j) in pts:
        row = odsg.kernel_row(g.astype(np.float64), rp, rs, h, (i, j))
        rows[(i, j)] = row
        got = host(planes[:, i, j])
        for k, (oy, ox) in enumerate(offs):
            want = row.get((i + oy, j + ox), 0.0)
            assert abs(got[k] - want) <= 1e-5 * want + 2e-7, (rp, rs, i, j, oy, ox, got[k], want)
    D.dsgnlm_balance(den, 0.0, 1)
    ones = torch.ones((256, 256), device="cuda")
    np.testing.assert_allclose(host(D.dsgnlm_apply(den, ones)), 1.0, atol=1e-6)
    # W z at sampled pixels from the oracle's rows: with d = g^(-1/2) (one update),
    # W_sr = d_s d_r K1_sr / m for r != s and the diagonal closed to a row sum of 1
    d, m = D.dsgnlm_copy_scaling(den)
    dh = host(d)
    z = np.random.default_rng(7).uniform(0, 1, (256, 256)).astype(np.float32)
    y = host(D.dsgnlm_apply(den, cuda(z)))
    for (i, j), row in rows.items():
        gs = sum(row.values())
        assert abs(dh[i, j] - gs ** -0.5) <= 1e-5 * gs ** -0.5
        off = {r: dh[i, j] * dh[r] * val / m for r, val in row.items() if r != (i, j)}
        want = sum(w * z[r] for r, w in off.items()) + (1.0 - sum(off.values())) * z[i, j]
        assert abs(y[i, j] - want) <= 1e-5 * abs(want) + 1e-6, (rp, rs, i, j)
