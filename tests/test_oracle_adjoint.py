"""The two FP64 references of the unrolled-solve derivatives agree: torch autograd on
the dense PyTorch form against central finite differences of the sparse NumPy
oracle, and the two forward losses against each other.  CPU only."""
import numpy as np
import pytest

import synthetic
from oracle import adjoint, problems

torch = pytest.importorskip("torch")


def _case(H=12, W=12, seed=5):
    wl = synthetic.workload("unroll8x256")
    inst = problems.sr_instance(wl, H=H, W=W, seed=seed)
    guide = np.clip(inst["x_true"] + 0.05 * np.random.default_rng(seed).standard_normal((H, W)), -0.05, 1.05)
    return wl, inst, guide.astype(np.float32).astype(np.float64)


def test_forward_losses_agree():
    wl, inst, guide = _case()
    a = adjoint.unrolled_loss(inst["y"], guide, 0.1, 1.0, inst["x_true"], 1, 2, 3, 4)
    b = adjoint.torch_unrolled_loss(inst["y"], guide, 0.1, 1.0, inst["x_true"], 1, 2, 3, 4).item()
    assert abs(a - b) <= 1e-13 * max(1.0, abs(a))


def test_autograd_matches_finite_differences():
    wl, inst, guide = _case()
    y = torch.tensor(inst["y"].astype(np.float64), requires_grad=True)
    g = torch.tensor(guide, requires_grad=True)
    h = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    rho = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    loss = adjoint.torch_unrolled_loss(y, g, h, rho, inst["x_true"], 1, 2, 3, 4)
    loss.backward()
    x_true = inst["x_true"]
    f_y = lambda yy: adjoint.unrolled_loss(yy, guide, 0.1, 1.0, x_true, 1, 2, 3, 4)
    f_g = lambda gg: adjoint.unrolled_loss(inst["y"], gg, 0.1, 1.0, x_true, 1, 2, 3, 4)
    for idx in [(0, 0), (2, 3), (5, 5)]:
        fd = adjoint.fd_gradient(f_y, inst["y"], idx, 1e-5)
        assert abs(fd - y.grad[idx].item()) <= 1e-6 + 1e-5 * abs(fd)
    for idx in [(0, 0), (4, 7), (11, 11), (6, 1)]:
        if not (0.02 < guide[idx] < 0.98):
            continue  # the clip of the initial state has a kink at 0 and 1
        fd = adjoint.fd_gradient(f_g, guide, idx, 1e-5)
        assert abs(fd - g.grad[idx].item()) <= 1e-6 + 1e-4 * abs(fd)
    fd_h = (adjoint.unrolled_loss(inst["y"], guide, 0.1 + 1e-6, 1.0, x_true, 1, 2, 3, 4)
            - adjoint.unrolled_loss(inst["y"], guide, 0.1 - 1e-6, 1.0, x_true, 1, 2, 3, 4)) / 2e-6
    assert abs(fd_h - h.grad.item()) <= 1e-6 + 1e-4 * abs(fd_h)
    fd_r = (adjoint.unrolled_loss(inst["y"], guide, 0.1, 1.0 + 1e-6, x_true, 1, 2, 3, 4)
            - adjoint.unrolled_loss(inst["y"], guide, 0.1, 1.0 - 1e-6, x_true, 1, 2, 3, 4)) / 2e-6
    assert abs(fd_r - rho.grad.item()) <= 1e-6 + 1e-4 * abs(fd_r)


def test_branch_trace_flags_steps_across_a_kink():
    # x0 = clip(guide, 0, 1): a guide pixel 0.5e-5 below 1 is inside the box, and a
    # step of +1e-5 moves it across the clip, so the traces differ; a step of the
    # same size on a pixel in the middle of the box changes no branch.
    wl, inst, guide = _case(8, 8, 3)
    g = np.clip(guide, 0.1, 0.9)
    g[2, 3] = 1.0 - 0.5e-5
    run = lambda gu: (lambda t: (adjoint.unrolled_loss(inst["y"], gu, 0.1, 1.0, inst["x_true"], 1, 2, 2, 3,
                                                       trace=t), t))({})
    _, base = run(g)
    assert len(base["clamp"]) == 3 and base["init"][2, 3] == 0
    up = g.copy()
    up[2, 3] += 1e-5
    _, t_up = run(up)
    assert t_up["init"][2, 3] == -1 and not adjoint.same_branches(base, t_up)
    mid = g.copy()
    mid[4, 4] += 1e-5
    _, t_mid = run(mid)
    assert adjoint.same_branches(base, t_mid)
