"""Single-photon imaging at the full 512x512 workload (4x4 sub-pixels, eta 4, 7x7
patches, 21x21 window, h 0.1, balance to 1e-6, 50 iterations, alpha 64) against the
full FP64 oracle solve, through the same pipeline calls as the benchmark."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import problems
from tests.gpu_helpers import cuda, host, rel_l2

pytestmark = pytest.mark.gpu


def test_spi_full_solve_matches_oracle(gpu_lib):
    from paper_1901_06110_gb300 import dsgnlm as D
    from paper_1901_06110_gb300 import pipeline
    wl = synthetic.workload("spi512")
    inst = problems.spi_instance(wl)
    # measurement made on the GPU must equal the oracle's bit for bit
    bits = D.lpnp_spi_observe(cuda(inst["x_true"]), cuda(inst["arrivals"]), wl["K_side"], wl["eta"])
    np.testing.assert_array_equal(host(bits), inst["bits"])
    counts = D.lpnp_spi_counts(bits, wl["K_side"])
    solver = pipeline.Solver(wl["H"], wl["W"], pipeline.Params.from_workload(wl), kind="spi")
    solver.run(counts)
    torch.cuda.synchronize()
    assert solver.balance[0] == 0
    ref = problems.solve_spi(wl, inst, tol=wl["tol"])
    assert rel_l2(host(solver.guide), ref["guide"]) <= 1e-6
    assert rel_l2(host(solver.x), ref["x"]) <= 1e-5
    assert rel_l2(host(solver.v), ref["v"]) <= 1e-5
