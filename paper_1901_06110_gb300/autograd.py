"""torch.autograd binding of the differentiable form (lpnp_unrolled_forward /
lpnp_backward and their batched forms in the C ABI): unrolled linearized PnP-ADMM for
2x super-resolution with DSG-NLM, differentiable in the observation, the guide, the
bandwidth h and rho.  Each image keeps a denoiser handle and a checkpoint tape between
the forward and the backward; these slots are pooled and reused once the backward has
run, so repeated calls allocate nothing.  The calls run on the caller's current stream.  All arithmetic runs in the
CUDA library."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _abi
from . import dsgnlm as D


@dataclass
class UnrollParams:
    patch_r: int = 2
    search_r: int = 7
    balance_passes: int = 4
    iters: int = 10
    alpha: float = 1.0
    blur_sigma: float = 1.0
    blur_r: int = 4


class _Slot:
    """One image's tape and FP32 denoiser handle.  The handle launches on the caller's
    current stream (set when it changes); the batched calls run every image of a batch
    in one launch per step on the first image's stream."""

    def __init__(self):
        self.lib = _abi.load()
        t = ctypes.c_void_p()
        D._check(self.lib.lpnp_tape_create(ctypes.byref(t)), "lpnp_tape_create")
        self.ptr = t
        self.den = D.dsgnlm_create("f32")
        self.bound = None  # the raw stream the handle launches on

    def bind(self, stream):
        raw = stream.cuda_stream
        if raw != self.bound:
            D._check(self.lib.dsgnlm_set_stream(self.den.handle, ctypes.c_void_p(raw)), "dsgnlm_set_stream")
            self.bound = raw

    def __del__(self):
        try:
            if self.ptr is not None and self.ptr.value:
                self.lib.lpnp_tape_destroy(self.ptr)
            self.den.close()
        except Exception:
            pass


_POOL: list[_Slot] = []


class _Lease:
    """Slots held by one recorded forward; they go back to the pool after the backward
    or when the autograd graph that holds the lease is freed."""

    def __init__(self, count: int):
        self.slots = [_POOL.pop() if _POOL else _Slot() for _ in range(count)]

    def release(self):
        # back in reverse, so that the next lease of the same size takes the same slots in
        # the same order (and the C calls replay the graphs recorded for them)
        _POOL.extend(reversed(self.slots))
        self.slots = []

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def _bind(slots):
    """Every slot's handle launches on the current stream, which is returned."""
    cur = torch.cuda.current_stream()
    for s in slots:
        s.bind(cur)
    return cur


def _follow(ctx):
    """The backward's stream: the current one, after the work the forward queued on its
    stream (the tapes are not tensors, so autograd does not order them)."""
    cur = torch.cuda.current_stream()
    if cur.cuda_stream != ctx.stream.cuda_stream:
        cur.wait_stream(ctx.stream)
    return cur


def _ptrs(vals):
    return (ctypes.c_void_p * len(vals))(*vals)


_SLOT_PTRS: dict = {}


def _slot_ptrs(slots):
    """The tape and handle address arrays of a slot sequence (built once per sequence)."""
    key = tuple(id(s) for s in slots)
    hit = _SLOT_PTRS.get(key)
    if hit is None or any(a is not b for a, b in zip(hit[0], slots)):
        hit = (tuple(slots), _ptrs([s.ptr.value for s in slots]), _ptrs([s.den.handle.value for s in slots]))
        _SLOT_PTRS[key] = hit
    return hit[1], hit[2]


def _rows(t):
    """The addresses of t[0], t[1], ... of a contiguous tensor, without indexing it."""
    base, step = t.data_ptr(), t[0].numel() * t.element_size()
    return _ptrs([base + b * step for b in range(t.shape[0])])


def _grad_scalar(ctx, idx, value):
    return torch.tensor(value, dtype=ctx.scalar_dtype[idx - 2]) if ctx.needs_input_grad[idx] else None


def _scalar_dtype(v):
    return v.dtype if isinstance(v, torch.Tensor) else torch.float64


class UnrolledSR(torch.autograd.Function):
    """x_N = unrolled_solve(y, guide, h, rho) for one image (y [H/2, W/2], guide [H, W])."""

    @staticmethod
    def forward(ctx, y, guide, h, rho, params: UnrollParams):
        y = y.detach().contiguous()
        guide = guide.detach().contiguous()
        H, W = guide.shape
        lease = _Lease(1)
        slot = lease.slots[0]
        x = torch.empty_like(guide)
        ctx.stream = _bind(lease.slots)
        D._check(slot.lib.lpnp_unrolled_forward(
            slot.ptr, slot.den.handle, D._ptr(y, torch.float32, "y", (H // 2) * (W // 2)),
            D._ptr(guide, torch.float32, "guide", H * W), H, W, params.patch_r, params.search_r, float(h),
            params.balance_passes, params.alpha, float(rho), params.iters, params.blur_sigma, params.blur_r,
            x.data_ptr()), "lpnp_unrolled_forward")
        ctx.lease = lease
        ctx.keep = (y, guide)  # the tape reads them in the backward
        ctx.scalar_dtype = (_scalar_dtype(h), _scalar_dtype(rho))
        return x

    @staticmethod
    def backward(ctx, x_bar):
        y, guide = ctx.keep
        slot = ctx.lease.slots[0]
        x_bar = x_bar.contiguous().float()
        y_bar = torch.empty_like(y)
        g_bar = torch.empty_like(guide)
        hb = ctypes.c_double(0.0)
        rb = ctypes.c_double(0.0)
        slot.bind(_follow(ctx))
        D._check(slot.lib.lpnp_backward(slot.ptr, x_bar.data_ptr(), y_bar.data_ptr(), g_bar.data_ptr(),
                                        ctypes.byref(hb), ctypes.byref(rb)), "lpnp_backward")
        ctx.lease.release()
        return y_bar, g_bar, _grad_scalar(ctx, 2, hb.value), _grad_scalar(ctx, 3, rb.value), None


class UnrolledSRBatch(torch.autograd.Function):
    """x_N [B, H, W] for y [B, H/2, W/2] and guide [B, H, W] with shared h and rho,
    through the batched C calls: every step is one launch over the B images."""

    @staticmethod
    def forward(ctx, y, guide, h, rho, params: UnrollParams):
        y = y.detach().contiguous()
        guide = guide.detach().contiguous()
        B, H, W = guide.shape
        if y.shape != (B, H // 2, W // 2) or y.dtype != torch.float32 or guide.dtype != torch.float32:
            raise ValueError("y must be float32 [B, H/2, W/2] and guide float32 [B, H, W]")
        lease = _Lease(B)
        x = torch.empty_like(guide)
        lib = lease.slots[0].lib
        ctx.stream = _bind(lease.slots)
        tapes, dens = _slot_ptrs(lease.slots)
        D._check(lib.lpnp_unrolled_forward_batched(
            tapes, dens, B, _rows(y), _rows(guide), H, W, params.patch_r, params.search_r, float(h),
            params.balance_passes, params.alpha, float(rho), params.iters, params.blur_sigma, params.blur_r,
            _rows(x)),
            "lpnp_unrolled_forward_batched")
        ctx.lease = lease
        ctx.keep = (y, guide)
        ctx.scalar_dtype = (_scalar_dtype(h), _scalar_dtype(rho))
        return x

    @staticmethod
    def backward(ctx, x_bar):
        y, guide = ctx.keep
        slots = ctx.lease.slots
        B = len(slots)
        x_bar = x_bar.contiguous().float()
        y_bar = torch.empty_like(y)
        g_bar = torch.empty_like(guide)
        hb = (ctypes.c_double * B)()
        rb = (ctypes.c_double * B)()
        cur = _follow(ctx)
        for s in slots:
            s.bind(cur)
        D._check(slots[0].lib.lpnp_backward_batched(
            _slot_ptrs(slots)[0], B, _rows(x_bar), _rows(y_bar), _rows(g_bar), hb, rb),
            "lpnp_backward_batched")
        ctx.lease.release()
        return y_bar, g_bar, _grad_scalar(ctx, 2, sum(hb)), _grad_scalar(ctx, 3, sum(rb)), None


def unrolled_sr(y, guide, h, rho, params: UnrollParams | None = None):
    """Batched: y [B, H/2, W/2], guide [B, H, W], h and rho scalars (tensors to receive
    gradients); returns x_N [B, H, W]."""
    return UnrolledSRBatch.apply(y, guide, h, rho, params or UnrollParams())
