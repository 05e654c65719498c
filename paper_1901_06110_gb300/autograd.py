"""torch.autograd binding of the differentiable form (lpnp_unrolled_forward /
lpnp_backward in the C ABI): unrolled linearized PnP-ADMM for 2x super-resolution
with DSG-NLM, differentiable in the observation, the guide, the bandwidth h and
rho.  Each image keeps its own denoiser handle and checkpoint tape between the
forward and the backward; all arithmetic runs in the CUDA library."""
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


class _Tape:
    def __init__(self):
        self.lib = _abi.load()
        t = ctypes.c_void_p()
        D._check(self.lib.lpnp_tape_create(ctypes.byref(t)), "lpnp_tape_create")
        self.ptr = t
        self.den = D.dsgnlm_create("f32")

    def __del__(self):
        try:
            if self.ptr is not None and self.ptr.value:
                self.lib.lpnp_tape_destroy(self.ptr)
            self.den.close()
        except Exception:
            pass


class UnrolledSR(torch.autograd.Function):
    """x_N = unrolled_solve(y, guide, h, rho) for one image."""

    @staticmethod
    def forward(ctx, y, guide, h, rho, params: UnrollParams):
        y = y.detach().contiguous()
        guide = guide.detach().contiguous()
        H, W = guide.shape
        tape = _Tape()
        x = torch.empty_like(guide)
        D._check(tape.lib.lpnp_unrolled_forward(
            tape.ptr, tape.den.handle, D._ptr(y, torch.float32, "y", (H // 2) * (W // 2)),
            D._ptr(guide, torch.float32, "guide", H * W), H, W, params.patch_r, params.search_r, float(h),
            params.balance_passes, params.alpha, float(rho), params.iters, params.blur_sigma, params.blur_r,
            x.data_ptr()), "lpnp_unrolled_forward")
        ctx.tape = tape
        ctx.keep = (y, guide)  # the tape reads them in the backward
        ctx.h_dtype = h.dtype if isinstance(h, torch.Tensor) else torch.float64
        return x

    @staticmethod
    def backward(ctx, x_bar):
        y, guide = ctx.keep
        x_bar = x_bar.contiguous().float()
        y_bar = torch.empty_like(y)
        g_bar = torch.empty_like(guide)
        hb = ctypes.c_double(0.0)
        rb = ctypes.c_double(0.0)
        D._check(ctx.tape.lib.lpnp_backward(ctx.tape.ptr, x_bar.data_ptr(), y_bar.data_ptr(), g_bar.data_ptr(),
                                            ctypes.byref(hb), ctypes.byref(rb)), "lpnp_backward")
        ctx.tape = None
        return (y_bar, g_bar, torch.tensor(hb.value, dtype=ctx.h_dtype),
                torch.tensor(rb.value, dtype=ctx.h_dtype), None)


def unrolled_sr(y, guide, h, rho, params: UnrollParams | None = None):
    """Batched convenience: y [B, H/2, W/2], guide [B, H, W], h and rho scalars
    (tensors to receive gradients); returns x_N [B, H, W]."""
    params = params or UnrollParams()
    outs = [UnrolledSR.apply(y[b], guide[b], h, rho, params) for b in range(guide.shape[0])]
    return torch.stack(outs)
