"""The allocation-free super-resolution gradient against the handle-based one.

lpnp_sr_gradient_noalloc exists for callers that cannot allocate device memory
when they need the gradient (for example a plugin whose host framework owns all
device allocations); it keeps its scratch in a fixed static device array.  Here it
is called through the C ABI, twice in a row with different inputs (the shared
scratch keeps the previous call's contents), and each result is compared with
lpnp_gradient on the same inputs.  The file is collected last so that a run that
stops at its first failure has run every other test already.
"""
import ctypes

import numpy as np
import pytest
import torch

import synthetic
from oracle import forward as ofw
from tests.gpu_helpers import cuda, host

pytestmark = pytest.mark.gpu


def _handle_gradient(x, y, blur_sigma, blur_r):
    from paper_1901_06110_gb300 import dsgnlm as D
    den = D.dsgnlm_create()
    p = D.Problem("sr", den, x.clone(), x.clone(), x.clone(), alpha=1.0, y=y, blur_sigma=blur_sigma,
                  blur_r=blur_r)
    g = D.lpnp_gradient(p, x)
    torch.cuda.synchronize()
    den.close()
    return g


def test_noalloc_gradient_matches_handle_gradient_twice(gpu_lib):
    from paper_1901_06110_gb300 import _abi
    stream = torch.cuda.current_stream().cuda_stream
    for call, (H, W, seed) in enumerate([(64, 96, 11), (46, 70, 12)]):
        x = cuda(synthetic.ground_truth(H, W, 6, True, seed))
        y = cuda(np.random.default_rng(seed).uniform(0, 1, (H // 2, W // 2)).astype(np.float32))
        g = torch.full((H, W), float("nan"), device="cuda")
        st = gpu_lib.lpnp_sr_gradient_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                              H, W, 1.0, 4, ctypes.c_void_p(g.data_ptr()),
                                              ctypes.c_void_p(stream))
        assert st == _abi.OK, (call, st)
        torch.cuda.synchronize()
        ref = _handle_gradient(x, y, 1.0, 4)
        np.testing.assert_allclose(host(g), host(ref), atol=1e-6, err_msg=f"call {call}")
        # and against the FP64 oracle, with the tolerance of the other gradient tests
        want = ofw.sr_grad(host(x), host(y), ofw.gaussian_psf(1.0, 4))
        np.testing.assert_allclose(host(g), want, atol=1e-6, err_msg=f"call {call}")


def test_noalloc_gradient_rejects_oversized_images(gpu_lib):
    from paper_1901_06110_gb300 import _abi
    # (H/2)(W/2) = 1024 * 1026 > 1,048,576: rejected before any launch (pointers unused)
    fake = ctypes.c_void_p(0x10000)
    st = gpu_lib.lpnp_sr_gradient_noalloc(fake, fake, 2048, 2052, 1.0, 4, fake, None)
    assert st == _abi.EINVAL


@pytest.mark.parametrize("H,W", [(2048, 2048), (4096, 1024)])
def test_noalloc_gradient_at_the_size_cap(gpu_lib, H, W):
    """(H/2)(W/2) = 1,048,576 exactly: the largest accepted size fills the whole
    array; every element of the result matches the handle-based gradient."""
    from paper_1901_06110_gb300 import _abi
    assert (H // 2) * (W // 2) == 1 << 20
    stream = torch.cuda.current_stream().cuda_stream
    x = cuda(synthetic.ground_truth(H, W, 6, True, 21))
    y = cuda(np.random.default_rng(21).uniform(0, 1, (H // 2, W // 2)).astype(np.float32))
    g = torch.full((H, W), float("nan"), device="cuda")
    st = gpu_lib.lpnp_sr_gradient_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), H, W,
                                          1.0, 4, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(stream))
    assert st == _abi.OK
    torch.cuda.synchronize()
    ref = _handle_gradient(x, y, 1.0, 4)
    np.testing.assert_allclose(host(g), host(ref), atol=1e-6)
