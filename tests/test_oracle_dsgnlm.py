"""Pins of the DSG-NLM oracle (Sec. 3) against brute force, closed forms and the
Theorem IV.1 invariants.  CPU only."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import dsgnlm


def _rand_guide(H, W, seed):
    return np.random.default_rng(seed).uniform(0, 1, (H, W))


@pytest.mark.parametrize("H,W,rp,rs,h", [(6, 7, 1, 2, 0.3), (5, 4, 2, 1, 0.5), (3, 8, 0, 3, 0.2),
                                         (4, 4, 3, 4, 0.7)])
def test_kernel_matches_brute_force(H, W, rp, rs, h):
    g = _rand_guide(H, W, H * 100 + W)
    K_fast = dsgnlm.kernel_matrix(g, rp, rs, h).toarray()
    K_bf = dsgnlm.brute_force_kernel(g, rp, rs, h)
    np.testing.assert_allclose(K_fast, K_bf, rtol=1e-13, atol=1e-15)


def test_two_pixel_row_closed_form():
    # 1x2 image [a, b], 3x3 patches, search radius 1.  With symmetric reflection
    # the two patches differ only in their middle column, in all three rows:
    # D = 3 (a - b)^2; N_p = 3, so k = exp(-3 (a-b)^2 / (2 * 9 * h^2)).
    # The hat at offset (0, 1) is (1 - 0)(1 - 1/2) = 1/2.
    a, b, h = 0.2, 0.5, 0.1
    k = math.exp(-3 * (a - b) ** 2 / (18 * h * h))
    q = 0.5 * k
    K1 = dsgnlm.kernel_matrix(np.array([[a, b]]), 1, 1, h).toarray()
    np.testing.assert_allclose(K1, [[1, q], [q, 1]], rtol=1e-14)
    # equal row sums: one Sinkhorn step balances exactly, m = 1, closure adds nothing
    d, k_upd, hist = dsgnlm.sinkhorn(sp.csr_matrix(K1), 1e-14, 50)
    W, m = dsgnlm.dsg_matrix(sp.csr_matrix(K1), d)
    np.testing.assert_allclose(W.toarray(), np.array([[1, q], [q, 1]]) / (1 + q), rtol=1e-14)
    assert abs(m - 1) < 1e-14


def test_two_pixel_column_closed_form():
    # the transposed layout (2x1) must give the same matrix
    a, b, h = 0.7, 0.1, 0.2
    k = math.exp(-3 * (a - b) ** 2 / (18 * h * h))
    K1 = dsgnlm.kernel_matrix(np.array([[a], [b]]), 1, 1, h).toarray()
    np.testing.assert_allclose(K1, [[1, 0.5 * k], [0.5 * k, 1]], rtol=1e-14)


def test_three_pixel_unequal_offsets():
    # 1x3 image, 1x1 patches (N_p = 1), search radius 2: hat at |o| = 1 is 2/3,
    # at |o| = 2 it is 1/3; D is the squared pixel difference.
    g = np.array([[0.1, 0.4, 0.9]])
    h = 0.3
    K1 = dsgnlm.kernel_matrix(g, 0, 2, h).toarray()
    kk = lambda u, v: math.exp(-(u - v) ** 2 / (2 * h * h))
    want = np.array([[1, 2 / 3 * kk(.1, .4), 1 / 3 * kk(.1, .9)],
                     [2 / 3 * kk(.4, .1), 1, 2 / 3 * kk(.4, .9)],
                     [1 / 3 * kk(.9, .1), 2 / 3 * kk(.9, .4), 1]])
    np.testing.assert_allclose(K1, want, rtol=1e-14)


def _check_theorem_iv1(W, tol):
    Wd = W.toarray()
    n = Wd.shape[0]
    np.testing.assert_allclose(Wd, Wd.T, atol=1e-15)
    np.testing.assert_allclose(Wd.sum(axis=1), np.ones(n), atol=tol)
    np.testing.assert_allclose(Wd.sum(axis=0), np.ones(n), atol=tol)
    assert (Wd >= -1e-15).all()
    ev = np.linalg.eigvalsh(Wd)
    assert ev.min() >= -1e-12 and ev.max() <= 1 + 1e-12
    assert abs(np.linalg.norm(Wd, 2) - 1) < 1e-12


@pytest.mark.parametrize("maxit", [1, 3, 10000])
def test_theorem_iv1_invariants(maxit):
    g = _rand_guide(9, 8, 7)
    W, info = dsgnlm.build_w(g, 1, 2, 0.25, 1e-13, maxit)
    _check_theorem_iv1(W, 1e-12)
    x = np.random.default_rng(3).uniform(0, 1, (9, 8))
    y = dsgnlm.denoise(W, x)
    assert abs(y.sum() - x.sum()) < 1e-11
    np.testing.assert_allclose(dsgnlm.denoise(W, np.full((9, 8), 0.37)), 0.37, atol=1e-14)


def test_sinkhorn_converges_and_step_one_is_eq_s2():
    g = _rand_guide(10, 9, 11)
    K1 = dsgnlm.kernel_matrix(g, 1, 3, 0.2)
    d1, k1, _ = dsgnlm.sinkhorn(K1, 0.0, 1)
    rowsum = np.asarray(K1.sum(axis=1)).ravel()
    assert k1 == 1
    np.testing.assert_allclose(d1, rowsum ** -0.5, rtol=1e-15)
    d, k, hist = dsgnlm.sinkhorn(K1, 1e-12, 10000)
    assert hist[-1] <= 1e-12 and k < 10000
    S = sp.diags(d) @ K1 @ sp.diags(d)
    np.testing.assert_allclose(np.asarray(S.sum(axis=1)).ravel(), 1, atol=1e-12)
    # converged balancing leaves m = 1 and a vanishing closure
    W, m = dsgnlm.dsg_matrix(K1, d)
    assert abs(m - 1) < 1e-11


@pytest.mark.parametrize("shape,rp,rs,h", [((5, 6), 1, 2, 0.3), ((4, 7), 2, 1, 0.15), ((6, 3), 0, 2, 0.4)])
def test_one_step_balance_equals_algorithm_2(shape, rp, rs, h):
    vt = _rand_guide(*shape, 5)
    want = dsgnlm.alg2_literal(vt, vt, rp, rs, h)
    W, _ = dsgnlm.build_w(vt, rp, rs, h, 0.0, 1)
    got = dsgnlm.denoise(W, vt)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-14)


def test_identity_special_cases():
    g = _rand_guide(7, 6, 9)
    x = _rand_guide(7, 6, 10)
    W0, _ = dsgnlm.build_w(g, 1, 0, 0.2, 1e-12, 100)  # search radius 0
    np.testing.assert_allclose(W0.toarray(), np.eye(42), atol=0)
    Wh, _ = dsgnlm.build_w(g, 1, 2, 1e-6, 1e-12, 100)  # vanishing bandwidth
    np.testing.assert_allclose(dsgnlm.denoise(Wh, x), x, atol=1e-15)


def test_constant_guide_is_hat_toeplitz():
    rs = 3
    g = np.full((12, 11), 0.42)
    K1 = dsgnlm.kernel_matrix(g, 2, rs, 0.1).toarray()
    rowsum = K1.sum(axis=1).reshape(12, 11)
    # an interior pixel sees the full window: (sum_a (1 - |a|/(rs+1)))^2 = (rs+1)^2
    assert abs(rowsum[6, 5] - (rs + 1) ** 2) < 1e-12
    s = 6 * 11 + 5
    for oy in range(-rs, rs + 1):
        for ox in range(-rs, rs + 1):
            r = (6 + oy) * 11 + 5 + ox
            assert abs(K1[s, r] - (1 - abs(oy) / (rs + 1)) * (1 - abs(ox) / (rs + 1))) < 1e-15


def test_sym_index():
    got = [int(dsgnlm.sym_index(i, 3)) for i in range(-7, 10)]
    # indices -7..9 of a 3-pixel row: ... 0 | 0 1 2 | 2 1 0 | 0 1 2 | 2 1 0 | 0 1 2 | 2 1 0 ...
    assert got == [0, 0, 1, 2, 2, 1, 0, 0, 1, 2, 2, 1, 0, 0, 1, 2, 2]


def test_kernel_row_matches_matrix():
    g = _rand_guide(11, 13, 21)
    K1 = dsgnlm.kernel_matrix(g, 2, 3, 0.2).tocsr()
    for s in [(0, 0), (5, 6), (10, 12), (3, 11)]:
        row = dsgnlm.kernel_row(g, 2, 3, 0.2, s)
        dense = K1[s[0] * 13 + s[1]].toarray().ravel()
        assert len(row) == np.count_nonzero(dense)
        for (ri, rj), val in row.items():
            assert abs(val - dense[ri * 13 + rj]) < 1e-15
