"""Thin PyTorch binding of the C ABI (include/dsgnlm.h).

Every function has the name of the C entry point it wraps and only marshals
arguments: tensors become device pointers, the current torch stream becomes the
CUDA stream, status codes become exceptions.  All arithmetic runs in the CUDA
library; when the library has not been built these functions raise.
"""
from __future__ import annotations

import ctypes

import torch

from . import _abi


class DsgnlmError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _abi.load()
        msg = lib.dsgnlm_strerror(status).decode()
        if status == _abi.ECUDA:
            msg += f" (cudaError {lib.dsgnlm_last_cuda_error()})"
        super().__init__(f"{where}: {msg} [status {status}]")
        self.status = status


def _check(status: int, where: str, ok=(_abi.OK,)):
    if status not in ok:
        raise DsgnlmError(status, where)
    return status


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _ptr(t: torch.Tensor, dtype: torch.dtype, name: str, numel: int | None = None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


_WDT = {"f32": _abi.F32, "f16": _abi.F16, "bf16": _abi.BF16}
_TORCH_WDT = {_abi.F32: torch.float32, _abi.F16: torch.float16, _abi.BF16: torch.bfloat16}


class Dsgnlm:
    """Owner of one dsgnlm_t handle (weight planes, scaling, scratch)."""

    def __init__(self, weight_dtype: str = "f32", stream=None):
        self.lib = _abi.load()
        self.wdtype = _WDT[weight_dtype]
        h = ctypes.c_void_p()
        _check(self.lib.dsgnlm_create(ctypes.byref(h), _stream(stream), self.wdtype), "dsgnlm_create")
        self.handle = h
        self.H = self.W = 0

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.dsgnlm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        _check(self.lib.dsgnlm_set_stream(self.handle, _stream(stream)), "dsgnlm_set_stream")


def dsgnlm_create(weight_dtype: str = "f32", stream=None) -> Dsgnlm:
    return Dsgnlm(weight_dtype, stream)


def dsgnlm_destroy(h: Dsgnlm) -> None:
    h.close()


def dsgnlm_build(h: Dsgnlm, guide: torch.Tensor, patch_r: int, search_r: int, bandwidth: float):
    H, W = guide.shape
    _check(h.lib.dsgnlm_build(h.handle, _ptr(guide, torch.float32, "guide"), H, W, patch_r,
                              search_r, float(bandwidth)), "dsgnlm_build")
    h.H, h.W = H, W


def dsgnlm_balance(h: Dsgnlm, tol: float, maxit: int):
    """Returns (status, updates, residual); status is OK, NOT_CONVERGED or STALLED."""
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    st = _check(h.lib.dsgnlm_balance(h.handle, float(tol), int(maxit), ctypes.byref(it), ctypes.byref(res)),
                "dsgnlm_balance", ok=(_abi.OK, _abi.NOT_CONVERGED, _abi.STALLED))
    return st, it.value, res.value


def dsgnlm_balance_batched(hs, tol: float, maxit: int, slices: int = 0):
    """Balance several built handles together (one phase-1 and one epilogue launch per
    pass over all of them).  slices = 0 keeps each handle's own offset schedule and
    gives each image exactly the dsgnlm_balance result; slices > 0 uses that many
    offset slices for every image.  Returns one (status, updates, residual) per handle."""
    count = len(hs)
    arr = (ctypes.c_void_p * count)(*[h.handle for h in hs])
    its = (ctypes.c_int * count)()
    res = (ctypes.c_double * count)()
    sts = (ctypes.c_int * count)()
    _check(_abi.load().dsgnlm_balance_batched(arr, count, float(tol), int(maxit), int(slices), its, res, sts),
           "dsgnlm_balance_batched")
    return [(sts[i], its[i], res[i]) for i in range(count)]


def dsgnlm_apply(h: Dsgnlm, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    n = h.H * h.W
    y = torch.empty_like(x) if out is None else out
    _check(h.lib.dsgnlm_apply(h.handle, _ptr(x, torch.float32, "x", n), _ptr(y, torch.float32, "y", n)),
           "dsgnlm_apply")
    return y


def dsgnlm_set_balance_scheme(h: Dsgnlm, scheme: str) -> None:
    """'sinkhorn' (plain symmetric Sinkhorn passes, the default) or 'accelerated'
    (two plain passes, then heavy-ball steps on log d; same fixed point)."""
    code = {"sinkhorn": _abi.BALANCE_SINKHORN, "accelerated": _abi.BALANCE_ACCELERATED}[scheme]
    _check(h.lib.dsgnlm_set_balance_scheme(h.handle, code), "dsgnlm_set_balance_scheme")


def dsgnlm_sync(h: Dsgnlm) -> int:
    """Wait for the handle's queued work; returns OK, or TIMEOUT if a bounded device
    wait gave up since the last report (the error word is then cleared)."""
    return _check(h.lib.dsgnlm_sync(h.handle), "dsgnlm_sync", ok=(_abi.OK, _abi.TIMEOUT))


def dsgnlm_set_wait_budget(h: Dsgnlm, cycles: int) -> None:
    """Cycles a stencil consumer waits for a weight tile (0: give up at once; a
    negative value restores the default of about 2 s)."""
    _check(h.lib.dsgnlm_set_wait_budget(h.handle, int(cycles)), "dsgnlm_set_wait_budget")


def dsgnlm_num_offsets(h: Dsgnlm) -> int:
    return h.lib.dsgnlm_num_offsets(h.handle)


def dsgnlm_copy_weights(h: Dsgnlm) -> torch.Tensor:
    nh = dsgnlm_num_offsets(h)
    dst = torch.empty((nh, h.H, h.W), dtype=_TORCH_WDT[h.wdtype], device="cuda")
    _check(h.lib.dsgnlm_copy_weights(h.handle, dst.data_ptr() if nh else None), "dsgnlm_copy_weights")
    return dst


def dsgnlm_copy_scaling(h: Dsgnlm):
    d = torch.empty((h.H, h.W), dtype=torch.float32, device="cuda")
    m = ctypes.c_double(0.0)
    _check(h.lib.dsgnlm_copy_scaling(h.handle, d.data_ptr(), ctypes.byref(m)), "dsgnlm_copy_scaling")
    return d, m.value


def _boundary(name: str) -> int:
    if name not in ("periodic", "symmetric"):
        raise ValueError(f"blur boundary must be 'periodic' or 'symmetric', got {name!r}")
    return _abi.BC_PERIODIC if name == "periodic" else _abi.BC_SYMMETRIC


def lpnp_sr_observe(x: torch.Tensor, noise: torch.Tensor | None, blur_sigma: float, blur_r: int,
                    out: torch.Tensor | None = None, boundary: str = "periodic") -> torch.Tensor:
    H, W = x.shape
    y = torch.empty((H // 2, W // 2), dtype=torch.float32, device=x.device) if out is None else out
    npt = None if noise is None else _ptr(noise, torch.float32, "noise", (H // 2) * (W // 2))
    _check(_abi.load().lpnp_sr_observe_bc(_ptr(x, torch.float32, "x"), npt, H, W, float(blur_sigma),
                                          int(blur_r), _boundary(boundary),
                                          _ptr(y, torch.float32, "y", (H // 2) * (W // 2)), _stream()),
           "lpnp_sr_observe_bc")
    return y


def lpnp_sr_guide(y: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    h, w = y.shape
    g = torch.empty((2 * h, 2 * w), dtype=torch.float32, device=y.device) if out is None else out
    _check(_abi.load().lpnp_sr_guide(_ptr(y, torch.float32, "y"), h, w,
                                     _ptr(g, torch.float32, "guide", 4 * h * w), _stream()), "lpnp_sr_guide")
    return g


def lpnp_spi_observe(x: torch.Tensor, arrivals: torch.Tensor, k_side: int, eta: float) -> torch.Tensor:
    H, W = x.shape
    bits = torch.empty((k_side * H, k_side * W), dtype=torch.uint8, device=x.device)
    _check(_abi.load().lpnp_spi_observe(_ptr(x, torch.float32, "x"),
                                        _ptr(arrivals, torch.float32, "arrivals", bits.numel()), H, W,
                                        int(k_side), float(eta), bits.data_ptr(), _stream()),
           "lpnp_spi_observe")
    return bits


def lpnp_spi_counts(bits: torch.Tensor, k_side: int) -> torch.Tensor:
    Hs, Ws = bits.shape
    H, W = Hs // k_side, Ws // k_side
    counts = torch.empty((H, W), dtype=torch.uint8, device=bits.device)
    _check(_abi.load().lpnp_spi_counts(_ptr(bits, torch.uint8, "bits"), H, W, int(k_side),
                                       counts.data_ptr(), _stream()), "lpnp_spi_counts")
    return counts


def lpnp_spi_guide(counts: torch.Tensor, K: int, eta: float) -> torch.Tensor:
    H, W = counts.shape
    g = torch.empty((H, W), dtype=torch.float32, device=counts.device)
    _check(_abi.load().lpnp_spi_guide(_ptr(counts, torch.uint8, "counts"), H, W, int(K), float(eta),
                                      g.data_ptr(), _stream()), "lpnp_spi_guide")
    return g


def lpnp_init(guide: torch.Tensor):
    """x = v = clip(guide, 0, 1), u = 0."""
    x = torch.empty_like(guide)
    v = torch.empty_like(guide)
    u = torch.empty_like(guide)
    _check(_abi.load().lpnp_init(_ptr(guide, torch.float32, "guide"), guide.numel(), x.data_ptr(),
                                 v.data_ptr(), u.data_ptr(), _stream()), "lpnp_init")
    return x, v, u


class Problem:
    """Python mirror of lpnp_problem; keeps the tensors it points to alive."""

    def __init__(self, kind: str, den: Dsgnlm, x, v, u, *, alpha: float, constraint: int = _abi.C_BOX01,
                 y=None, blur_sigma: float = 1.0, blur_r: int = 4, counts=None, K: int = 16,
                 eta: float = 4.0, spi_eps: float = 1e-3, boundary: str = "periodic"):
        H, W = x.shape
        self.den, self.x, self.v, self.u, self.y, self.counts = den, x, v, u, y, counts
        s = _abi.LpnpProblem()
        s.kind = _abi.SR2 if kind == "sr" else _abi.SPI
        s.H, s.W = H, W
        s.y = _ptr(y, torch.float32, "y", (H // 2) * (W // 2)) if y is not None else None
        s.blur_sigma, s.blur_r = float(blur_sigma), int(blur_r)
        s.counts = _ptr(counts, torch.uint8, "counts", H * W) if counts is not None else None
        s.K, s.eta, s.spi_eps = int(K), float(eta), float(spi_eps)
        s.constraint, s.alpha = int(constraint), float(alpha)
        s.den = den.handle.value if den is not None else None
        s.x = _ptr(x, torch.float32, "x", H * W)
        s.v = _ptr(v, torch.float32, "v", H * W)
        s.u = _ptr(u, torch.float32, "u", H * W)
        s.resid_hist = None
        s.blur_boundary = _boundary(boundary)
        self.struct = s


def lpnp_gradient(p: Problem, x: torch.Tensor) -> torch.Tensor:
    g = torch.empty_like(x)
    _check(_abi.load().lpnp_gradient(ctypes.byref(p.struct), _ptr(x, torch.float32, "x"),
                                     g.data_ptr()), "lpnp_gradient")
    return g


def lpnp_sr_gradient_noalloc(x: torch.Tensor, y: torch.Tensor, blur_sigma: float, blur_r: int,
                             out: torch.Tensor | None = None) -> torch.Tensor:
    """A^T (A x - y) with the periodic blur, without any device allocation inside the
    call (its scratch is a fixed 4 MiB array shared by all calls on the device; see
    include/dsgnlm.h).  Equal to lpnp_gradient only for problems whose blur boundary
    is periodic; not for use on a device after a device reset."""
    H, W = x.shape
    g = torch.empty_like(x) if out is None else out
    _check(_abi.load().lpnp_sr_gradient_noalloc(_ptr(x, torch.float32, "x"),
                                                _ptr(y, torch.float32, "y", (H // 2) * (W // 2)), H, W,
                                                float(blur_sigma), int(blur_r),
                                                _ptr(g, torch.float32, "grad", H * W), _stream()),
           "lpnp_sr_gradient_noalloc")
    return g


def lpnp_solve(p: Problem, rho: float, iters: int, residuals: bool = False):
    """Run Algorithm 1 in place on p.x, p.v, p.u.  With residuals=True returns the
    per-iteration (primal, dual) RMS residuals as a list of pairs."""
    hist = (ctypes.c_double * (2 * iters))() if residuals and iters > 0 else None
    p.struct.resid_hist = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double)) if hist is not None else None
    try:
        _check(_abi.load().lpnp_solve(ctypes.byref(p.struct), float(rho), int(iters)), "lpnp_solve")
    finally:
        p.struct.resid_hist = None
    if hist is None:
        return None
    return [(hist[2 * k], hist[2 * k + 1]) for k in range(iters)]


def lpnp_solve_standard(p: Problem, rho: float, iters: int, cg_iters: int, residuals: bool = False):
    """Standard PnP-ADMM (SR): the x-update takes cg_iters conjugate-gradient steps on
    (A^T A + rho I) x = A^T y + rho (v - u) from the current x, then projects."""
    hist = (ctypes.c_double * (2 * iters))() if residuals and iters > 0 else None
    p.struct.resid_hist = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double)) if hist is not None else None
    try:
        _check(_abi.load().lpnp_solve_standard(ctypes.byref(p.struct), float(rho), int(iters), int(cg_iters)),
               "lpnp_solve_standard")
    finally:
        p.struct.resid_hist = None
    if hist is None:
        return None
    return [(hist[2 * k], hist[2 * k + 1]) for k in range(iters)]


def lpnp_solve_adaptive(p: Problem, rho: float, iters: int, adapt_iters: int, patch_r: int, search_r: int,
                        bandwidth: float, tol: float, maxit: int, residuals: bool = False):
    """Algorithm 1 with W rebuilt from x + u in the first adapt_iters iterations
    (A-DSG-NLM when adapt_iters >= iters, the adapt-then-freeze F-DSG-NLM schedule
    otherwise).  p.den need not be built; it holds the last W afterwards."""
    hist = (ctypes.c_double * (2 * iters))() if residuals and iters > 0 else None
    p.struct.resid_hist = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double)) if hist is not None else None
    try:
        _check(_abi.load().lpnp_solve_adaptive(ctypes.byref(p.struct), float(rho), int(iters), int(adapt_iters),
                                               int(patch_r), int(search_r), float(bandwidth), float(tol),
                                               int(maxit)), "lpnp_solve_adaptive")
        p.den.H, p.den.W = p.struct.H, p.struct.W  # the handle now holds a W of this size
    finally:
        p.struct.resid_hist = None
    if hist is None:
        return None
    return [(hist[2 * k], hist[2 * k + 1]) for k in range(iters)]


def dsgnlm_profile_enable(h: Dsgnlm, enable: bool = True) -> None:
    _check(h.lib.dsgnlm_profile_enable(h.handle, int(bool(enable))), "dsgnlm_profile_enable")


def dsgnlm_profile_read(h: Dsgnlm, kind: int):
    """(total milliseconds, launches) of one timed kernel kind."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int(0)
    _check(h.lib.dsgnlm_profile_read(h.handle, int(kind), ctypes.byref(ms), ctypes.byref(n)),
           "dsgnlm_profile_read")
    return ms.value, n.value


def lpnp_tune_batched(problems, rho: float, candidates=(0, 1, 2, 3, 4), trial_iters: int = 2):
    """Time the batch under each candidate offset schedule (on copies of the
    iterates) and return (best slices, {slices: ms per iteration})."""
    count = len(problems)
    arr = (_abi.LpnpProblem * count)()
    for i, p in enumerate(problems):
        arr[i] = p.struct
        arr[i].resid_hist = None
    cand = (ctypes.c_int * len(candidates))(*[int(c) for c in candidates])
    ms = (ctypes.c_float * len(candidates))()
    best = ctypes.c_int(-1)
    _check(_abi.load().lpnp_tune_batched(arr, count, float(rho), cand, len(candidates), int(trial_iters),
                                         ctypes.byref(best), ms), "lpnp_tune_batched")
    return best.value, {int(c): float(ms[k]) for k, c in enumerate(candidates)}


def lpnp_solve_batched(problems, rho: float, iters: int, residuals: bool = False, slices: int | None = None):
    """Algorithm 1 for several images at once (one launch per step over all of
    them; the step sequence is replayed from a CUDA graph).  `slices` selects the
    offset schedule (None or 0: each handle's own plan).  Returns per-problem
    residual lists when residuals=True."""
    count = len(problems)
    arr = (_abi.LpnpProblem * count)()
    hists = []
    for i, p in enumerate(problems):
        arr[i] = p.struct
        if residuals and iters > 0:
            h = (ctypes.c_double * (2 * iters))()
            hists.append(h)
            arr[i].resid_hist = ctypes.cast(h, ctypes.POINTER(ctypes.c_double))
        else:
            arr[i].resid_hist = None
    if slices:
        _check(_abi.load().lpnp_solve_batched_sched(arr, count, float(rho), int(iters), int(slices)),
               "lpnp_solve_batched_sched")
    else:
        _check(_abi.load().lpnp_solve_batched(arr, count, float(rho), int(iters)), "lpnp_solve_batched")
    if not hists:
        return None
    return [[(h[2 * k], h[2 * k + 1]) for k in range(iters)] for h in hists]


def dsgnlm_launch_count() -> int:
    return int(_abi.load().dsgnlm_launch_count())


def dsgnlm_is_checked() -> bool:
    """True when the loaded library is the checked build (-DDSGNLM_CHECKED)."""
    return bool(_abi.load().dsgnlm_is_checked())


def dsgnlm_check_word(clear: bool = False) -> int:
    """The checked build's index-check word (0: no access left its buffer)."""
    w = ctypes.c_uint(0)
    _check(_abi.load().dsgnlm_check_word(ctypes.byref(w), int(bool(clear))), "dsgnlm_check_word")
    return int(w.value)


def dsgnlm_check_selftest(index: int, bound: int) -> None:
    """Run the checked build's index test once on (index, bound), touching no buffer."""
    _check(_abi.load().dsgnlm_check_selftest(int(index), int(bound)), "dsgnlm_check_selftest")
