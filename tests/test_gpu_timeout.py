"""The bounded waits of the stencil kernels report DSGNLM_TIMEOUT without a fault
or a hang, and leave the handle usable.

dsgnlm_set_wait_budget(h, 0) makes every consumer of the phase-1 kernel give up
at its first wait for a weight tile, as if the copy had not landed in time: the
CTA sets the handle's error word, the producer stops issuing copies and waits for
those in flight, and the kernel returns.  The test then checks that the failure
is reported once (dsgnlm_sync, dsgnlm_balance), that the error word is cleared by
the report, and that with the default budget restored the same handle gives the
earlier results bit for bit and matches the FP64 oracle (Algorithm 2's third
aggregation with the W of Eqs. S1-S3)."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import dsgnlm as odsg
from tests.gpu_helpers import cuda, host, rel_l2

pytestmark = pytest.mark.gpu


def test_apply_and_balance_time_out_and_recover(gpu_lib):
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    H, W, rp, rs, h = 48, 72, 2, 5, 0.1
    guide = synthetic.ground_truth(H, W, 8, True, 61)
    den = D.dsgnlm_create("f32")
    D.dsgnlm_build(den, cuda(guide), rp, rs, h)
    st0 = D.dsgnlm_balance(den, 1e-6, 200)
    assert st0[0] == _abi.OK
    d0, m0 = D.dsgnlm_copy_scaling(den)
    z = cuda(np.random.default_rng(7).uniform(0, 1, (H, W)).astype(np.float32))
    y0 = host(D.dsgnlm_apply(den, z))
    assert D.dsgnlm_sync(den) == _abi.OK

    # every consumer gives up at its first wait: the apply reports TIMEOUT once
    D.dsgnlm_set_wait_budget(den, 0)
    D.dsgnlm_apply(den, z)
    assert D.dsgnlm_sync(den) == _abi.TIMEOUT
    assert D.dsgnlm_sync(den) == _abi.OK  # the report cleared the error word
    # a balance under the same budget ends (bounded by maxit) and reports TIMEOUT
    with pytest.raises(D.DsgnlmError) as e:
        D.dsgnlm_balance(den, 1e-6, 20)
    assert e.value.status == _abi.TIMEOUT

    # default budget again: the same handle balances and applies as before
    D.dsgnlm_set_wait_budget(den, -1)
    assert D.dsgnlm_balance(den, 1e-6, 200) == st0
    d1, m1 = D.dsgnlm_copy_scaling(den)
    assert m1 == m0
    np.testing.assert_array_equal(host(d1), host(d0))
    y1 = host(D.dsgnlm_apply(den, z))
    assert D.dsgnlm_sync(den) == _abi.OK
    np.testing.assert_array_equal(y1, y0)
    Wm, _ = odsg.build_w(guide.astype(np.float64), rp, rs, h, 1e-6, 200)
    want = odsg.denoise(Wm, host(z))
    assert rel_l2(y1, want) <= 1e-5
    den.close()


def test_wait_budget_arguments(gpu_lib):
    from paper_1901_06110_gb300 import _abi
    from paper_1901_06110_gb300 import dsgnlm as D
    den = D.dsgnlm_create("f32")
    with pytest.raises(D.DsgnlmError) as e:
        D.dsgnlm_set_wait_budget(den, 4_000_000_001)  # above the default: refused
    assert e.value.status == _abi.EINVAL
    D.dsgnlm_set_wait_budget(den, 1000)
    D.dsgnlm_set_wait_budget(den, -5)
    assert D.dsgnlm_sync(den) == _abi.OK  # nothing queued, no error word yet
    den.close()
