"""The restoration experiments of Sec. 4 as sequences of C ABI calls.

One call of ``solve_sr`` / ``solve_spi`` is one pass of the whole method on one
image: guide from the measurements, weight build (Eq. NLM, S1), balance (Eq. S2,
S3), then Algorithm 1 with the fixed DSG-NLM (F-DSG-NLM) as denoiser.  Only
argument marshalling happens here; each step is a kernel of the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import _abi
from . import dsgnlm as D


@dataclass
class Params:
    patch_r: int
    search_r: int
    h: float
    tol: float
    iters: int
    rho: float = 1.0
    alpha: float = 1.0
    maxit: int = 10000
    blur_sigma: float = 1.0
    blur_r: int = 4
    K: int = 16
    eta: float = 4.0
    spi_eps: float = 1e-3
    weight_dtype: str = "f32"
    boundary: str = "periodic"  # SR blur boundary: "periodic" or "symmetric"
    # balance update rule: "accelerated" (heavy-ball passes after two plain ones; the
    # same fixed point in fewer passes) or "sinkhorn" (plain passes)
    balance: str = "accelerated"
    extra: dict = field(default_factory=dict)

    @staticmethod
    def from_workload(wl: dict, **over) -> "Params":
        keys = ("patch_r", "search_r", "h", "tol", "iters", "rho", "alpha", "blur_sigma", "blur_r",
                "eta", "spi_eps", "boundary")
        kw = {k: wl[k] for k in keys if k in wl}
        if "K_side" in wl:
            kw["K"] = wl["K_side"] ** 2
        kw.update(over)
        return Params(**kw)


class Solver:
    """Holds one denoiser handle and the iterate buffers for repeated solves of
    same-sized problems (buffers are reused, nothing is reallocated per call)."""

    def __init__(self, H: int, W: int, params: Params, kind: str = "sr"):
        self.H, self.W, self.p, self.kind = H, W, params, kind
        self.den = D.dsgnlm_create(params.weight_dtype)
        D.dsgnlm_set_balance_scheme(self.den, params.balance)
        self.x = torch.empty((H, W), device="cuda")
        self.v = torch.empty_like(self.x)
        self.u = torch.empty_like(self.x)
        self.guide = torch.empty_like(self.x)
        self.balance = None
        self._prob = None
        self._data = None

    def _problem(self, data):
        if self._prob is None or self._data is not data:
            p = self.p
            if self.kind == "sr":
                self._prob = D.Problem("sr", self.den, self.x, self.v, self.u, alpha=p.alpha, y=data,
                                       blur_sigma=p.blur_sigma, blur_r=p.blur_r, boundary=p.boundary)
            else:
                self._prob = D.Problem("spi", self.den, self.x, self.v, self.u, alpha=p.alpha,
                                       counts=data, K=p.K, eta=p.eta, spi_eps=p.spi_eps)
            self._data = data
        return self._prob

    def run(self, data: torch.Tensor, residuals: bool = False):
        """data: the [H/2][W/2] FP32 observation (SR) or the [H][W] uint8 counts (SPI)."""
        p = self.p
        lib = _abi.load()
        stream = D._stream()
        if self.kind == "sr":
            D._check(lib.lpnp_sr_guide(data.data_ptr(), self.H // 2, self.W // 2, self.guide.data_ptr(),
                                       stream), "lpnp_sr_guide")
        else:
            D._check(lib.lpnp_spi_guide(data.data_ptr(), self.H, self.W, p.K, p.eta, self.guide.data_ptr(),
                                        stream), "lpnp_spi_guide")
        D.dsgnlm_build(self.den, self.guide, p.patch_r, p.search_r, p.h)
        # the initial state does not depend on the balance, which ends with a host
        # synchronisation: queue it first, so that only the solve follows the wait
        D._check(lib.lpnp_init(self.guide.data_ptr(), self.H * self.W, self.x.data_ptr(),
                               self.v.data_ptr(), self.u.data_ptr(), stream), "lpnp_init")
        self.balance = D.dsgnlm_balance(self.den, p.tol, p.maxit)
        return D.lpnp_solve(self._problem(data), p.rho, p.iters, residuals=residuals)

    def prepare(self, data: torch.Tensor):
        """Guide, weight build, balance and the initial state (the part of run before
        Algorithm 1)."""
        p = self.p
        lib = _abi.load()
        stream = D._stream()
        if self.kind == "sr":
            D._check(lib.lpnp_sr_guide(data.data_ptr(), self.H // 2, self.W // 2, self.guide.data_ptr(),
                                       stream), "lpnp_sr_guide")
        else:
            D._check(lib.lpnp_spi_guide(data.data_ptr(), self.H, self.W, p.K, p.eta, self.guide.data_ptr(),
                                        stream), "lpnp_spi_guide")
        D.dsgnlm_build(self.den, self.guide, p.patch_r, p.search_r, p.h)
        self.balance = D.dsgnlm_balance(self.den, p.tol, p.maxit)
        D._check(lib.lpnp_init(self.guide.data_ptr(), self.H * self.W, self.x.data_ptr(),
                               self.v.data_ptr(), self.u.data_ptr(), stream), "lpnp_init")

    def run_standard(self, data: torch.Tensor, cg_iters: int, iters: int | None = None, residuals: bool = False):
        """Standard PnP-ADMM on the same W (SR): each x-update takes cg_iters
        conjugate-gradient steps.  Continues from the current state; call prepare
        first for a fresh solve."""
        return D.lpnp_solve_standard(self._problem(data), self.p.rho, self.p.iters if iters is None else iters,
                                     cg_iters, residuals=residuals)

    def run_adaptive(self, data: torch.Tensor, adapt_iters: int, residuals: bool = False):
        """The same solve with W rebuilt from x + u in the first adapt_iters
        iterations (Sec. 4): A-DSG-NLM when adapt_iters >= iters, otherwise the
        adapt-then-freeze F-DSG-NLM schedule.  The guide only sets the initial state."""
        p = self.p
        lib = _abi.load()
        stream = D._stream()
        if self.kind == "sr":
            D._check(lib.lpnp_sr_guide(data.data_ptr(), self.H // 2, self.W // 2, self.guide.data_ptr(),
                                       stream), "lpnp_sr_guide")
        else:
            D._check(lib.lpnp_spi_guide(data.data_ptr(), self.H, self.W, p.K, p.eta, self.guide.data_ptr(),
                                        stream), "lpnp_spi_guide")
        D._check(lib.lpnp_init(self.guide.data_ptr(), self.H * self.W, self.x.data_ptr(),
                               self.v.data_ptr(), self.u.data_ptr(), stream), "lpnp_init")
        hist = D.lpnp_solve_adaptive(self._problem(data), p.rho, p.iters, adapt_iters, p.patch_r, p.search_r, p.h,
                                     p.tol, p.maxit, residuals=residuals)
        self.balance = None
        return hist

    def close(self):
        self.den.close()


class BatchSolver:
    """Many super-resolution images of uneven sizes solved together: per image a
    guide, weight build and balance, then Algorithm 1 for all images at once with
    lpnp_solve_batched (one launch per step over all images, replayed from a CUDA
    graph), under the offset schedule `slices` that tune() picks by measurement."""

    def __init__(self, shapes, params: Params):
        self.p = params
        self.shapes = list(shapes)
        self.dens = [D.dsgnlm_create(params.weight_dtype) for _ in self.shapes]
        for d in self.dens:
            D.dsgnlm_set_balance_scheme(d, params.balance)
        self.x = [torch.empty(s, device="cuda") for s in self.shapes]
        self.v = [torch.empty_like(t) for t in self.x]
        self.u = [torch.empty_like(t) for t in self.x]
        self.guide = [torch.empty_like(t) for t in self.x]
        self.balance = [None] * len(self.shapes)
        self.slices = 0  # offset schedule of the batched steps (0: each handle's own plan)
        self.tuning = None
        self._probs = None
        self._ys = None

    def _problems(self, ys):
        p = self.p
        if self._probs is None or self._ys is not ys:
            self._probs = [D.Problem("sr", self.dens[i], self.x[i], self.v[i], self.u[i], alpha=p.alpha, y=ys[i],
                                     blur_sigma=p.blur_sigma, blur_r=p.blur_r) for i in range(len(self.shapes))]
            self._ys = ys
        return self._probs

    def tune(self, ys, candidates=(0, 1, 2, 3, 4), trial_iters: int = 2):
        """Pick the batched offset schedule by timing each candidate on this batch
        (the weights must be built and balanced: call after run, or prepare first)."""
        self.slices, self.tuning = D.lpnp_tune_batched(self._problems(ys), self.p.rho, candidates, trial_iters)
        return self.slices

    def prepare(self, ys):
        """Guide and weight build of every image, one batched balance of all of them
        under the batch's offset schedule (with the default, each handle's own plan,
        each image's result is that of its own dsgnlm_balance), and the initial state."""
        p = self.p
        lib = _abi.load()
        stream = D._stream()
        for i, (H, W) in enumerate(self.shapes):
            D._check(lib.lpnp_sr_guide(ys[i].data_ptr(), H // 2, W // 2, self.guide[i].data_ptr(), stream),
                     "lpnp_sr_guide")
            D.dsgnlm_build(self.dens[i], self.guide[i], p.patch_r, p.search_r, p.h)
        self.balance = D.dsgnlm_balance_batched(self.dens, p.tol, p.maxit, self.slices)
        for i, (H, W) in enumerate(self.shapes):
            D._check(lib.lpnp_init(self.guide[i].data_ptr(), H * W, self.x[i].data_ptr(), self.v[i].data_ptr(),
                                   self.u[i].data_ptr(), stream), "lpnp_init")

    def run(self, ys, residuals: bool = False):
        self.prepare(ys)
        return D.lpnp_solve_batched(self._problems(ys), self.p.rho, self.p.iters, residuals=residuals,
                                    slices=self.slices)

    def close(self):
        for d in self.dens:
            d.close()
