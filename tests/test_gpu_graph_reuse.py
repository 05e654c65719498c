"""The single-image solve is recorded as a CUDA graph and replayed.  1/m of the
balanced W is read on the device, so images of one size with different W replay the
same graphs (two are kept, one per parity of the balance's pass count).  A handle
that solves several images in turn gives each exactly the result of a fresh handle."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import problems
from tests.gpu_helpers import cuda, host

pytestmark = pytest.mark.gpu


def test_solve_graphs_replayed_across_images(gpu_lib):
    from paper_1901_06110_gb300 import pipeline
    wl = dict(synthetic.workload("sr64"), search_r=5, tol=1e-6)
    H, W = 64, 96
    insts = [problems.sr_instance(wl, H=H, W=W, seed=s) for s in (3, 4, 5)]
    params = pipeline.Params.from_workload(wl, iters=6)
    ref = []
    for inst in insts:
        s = pipeline.Solver(H, W, params)
        s.run(cuda(inst["y"]))
        torch.cuda.synchronize()
        ref.append((host(s.x), host(s.v), host(s.u)))
    shared = pipeline.Solver(H, W, params)
    for idx in (0, 1, 0, 2, 1, 2, 0):
        shared.run(cuda(insts[idx]["y"]))
        torch.cuda.synchronize()
        for got, want in zip((host(shared.x), host(shared.v), host(shared.u)), ref[idx]):
            assert np.array_equal(got, want)
