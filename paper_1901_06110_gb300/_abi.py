"""ctypes declarations of the C ABI in include/dsgnlm.h (no logic beyond loading)."""
from __future__ import annotations

import ctypes
import os

from .build import LIB_PATH

c_int, c_float, c_double, c_void_p = ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_void_p

# status codes
OK, EINVAL, ENOMEM, ECUDA, NOT_BUILT, NOT_BALANCED, NOT_CONVERGED, STALLED, TIMEOUT = range(9)
F32, F16, BF16 = 0, 1, 2
SR2, SPI = 0, 1
C_NONE, C_NONNEG, C_BOX01 = 0, 1, 2
BC_PERIODIC, BC_SYMMETRIC = 0, 1
MAX_PATCH_R, MAX_SEARCH_R = 14, 24
PROF_BUILD, PROF_BALANCE, PROF_APPLY, PROF_XUPDATE = range(4)
BALANCE_SINKHORN, BALANCE_ACCELERATED = 0, 1


class LpnpProblem(ctypes.Structure):
    _fields_ = [
        ("kind", c_int), ("H", c_int), ("W", c_int),
        ("y", c_void_p), ("blur_sigma", c_float), ("blur_r", c_int),
        ("counts", c_void_p), ("K", c_int), ("eta", c_float), ("spi_eps", c_float),
        ("constraint", c_int), ("alpha", c_float), ("den", c_void_p),
        ("x", c_void_p), ("v", c_void_p), ("u", c_void_p),
        ("resid_hist", ctypes.POINTER(c_double)),
        ("blur_boundary", c_int),
    ]


# name -> (restype, argtypes), exactly the functions declared in include/dsgnlm.h
SIGNATURES = {
    "dsgnlm_create": (c_int, [ctypes.POINTER(c_void_p), c_void_p, c_int]),
    "dsgnlm_destroy": (None, [c_void_p]),
    "dsgnlm_set_stream": (c_int, [c_void_p, c_void_p]),
    "dsgnlm_build": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_float]),
    "dsgnlm_balance": (c_int, [c_void_p, c_double, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_double)]),
    "dsgnlm_balance_batched": (c_int, [ctypes.POINTER(c_void_p), c_int, c_double, c_int, c_int,
                                       ctypes.POINTER(c_int), ctypes.POINTER(c_double), ctypes.POINTER(c_int)]),
    "dsgnlm_apply": (c_int, [c_void_p, c_void_p, c_void_p]),
    "dsgnlm_sync": (c_int, [c_void_p]),
    "dsgnlm_set_balance_scheme": (c_int, [c_void_p, c_int]),
    "dsgnlm_set_wait_budget": (c_int, [c_void_p, ctypes.c_longlong]),
    "dsgnlm_copy_weights": (c_int, [c_void_p, c_void_p]),
    "dsgnlm_copy_scaling": (c_int, [c_void_p, c_void_p, ctypes.POINTER(c_double)]),
    "dsgnlm_num_offsets": (c_int, [c_void_p]),
    "lpnp_sr_observe": (c_int, [c_void_p, c_void_p, c_int, c_int, c_float, c_int, c_void_p, c_void_p]),
    "lpnp_sr_observe_bc": (c_int, [c_void_p, c_void_p, c_int, c_int, c_float, c_int, c_int, c_void_p, c_void_p]),
    "lpnp_sr_guide": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "lpnp_spi_observe": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_float, c_void_p, c_void_p]),
    "lpnp_spi_counts": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]),
    "lpnp_spi_guide": (c_int, [c_void_p, c_int, c_int, c_int, c_float, c_void_p, c_void_p]),
    "lpnp_init": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lpnp_gradient": (c_int, [ctypes.POINTER(LpnpProblem), c_void_p, c_void_p]),
    "lpnp_solve": (c_int, [ctypes.POINTER(LpnpProblem), c_float, c_int]),
    "lpnp_solve_standard": (c_int, [ctypes.POINTER(LpnpProblem), c_float, c_int, c_int]),
    "lpnp_solve_adaptive": (c_int, [ctypes.POINTER(LpnpProblem), c_float, c_int, c_int, c_int, c_int, c_float,
                                    c_double, c_int]),
    "lpnp_solve_batched": (c_int, [ctypes.POINTER(LpnpProblem), c_int, c_float, c_int]),
    "lpnp_solve_batched_sched": (c_int, [ctypes.POINTER(LpnpProblem), c_int, c_float, c_int, c_int]),
    "lpnp_tune_batched": (c_int, [ctypes.POINTER(LpnpProblem), c_int, c_float, ctypes.POINTER(c_int), c_int, c_int,
                                  ctypes.POINTER(c_int), ctypes.POINTER(c_float)]),
    "lpnp_sr_gradient_noalloc": (c_int, [c_void_p, c_void_p, c_int, c_int, c_float, c_int, c_void_p,
                                         c_void_p]),
    "lpnp_tape_create": (c_int, [ctypes.POINTER(c_void_p)]),
    "lpnp_tape_destroy": (None, [c_void_p]),
    "lpnp_unrolled_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_float,
                                      c_int, c_float, c_float, c_int, c_float, c_int, c_void_p]),
    "lpnp_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double),
                              ctypes.POINTER(c_double)]),
    "lpnp_unrolled_forward_batched": (c_int, [ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_int,
                                              ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_int, c_int,
                                              c_int, c_int, c_float, c_int, c_float, c_float, c_int, c_float,
                                              c_int, ctypes.POINTER(c_void_p)]),
    "lpnp_backward_batched": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(c_void_p),
                                      ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), ctypes.POINTER(c_double),
                                      ctypes.POINTER(c_double)]),
    "dsgnlm_profile_enable": (c_int, [c_void_p, c_int]),
    "dsgnlm_profile_read": (c_int, [c_void_p, c_int, ctypes.POINTER(c_double), ctypes.POINTER(c_int)]),
    "dsgnlm_launch_count": (ctypes.c_uint64, []),
    "dsgnlm_last_cuda_error": (c_int, []),
    "dsgnlm_strerror": (ctypes.c_char_p, [c_int]),
    "dsgnlm_is_checked": (c_int, []),
    "dsgnlm_check_word": (c_int, [ctypes.POINTER(ctypes.c_uint), c_int]),
    "dsgnlm_check_selftest": (c_int, [ctypes.c_longlong, ctypes.c_longlong]),
}

_lib = None


def default_path() -> str:
    """The library this process uses: ``$DSGNLM_LIBRARY`` if set (for example the
    checked build), else ``lib/libdsgnlm.so``."""
    return os.environ.get("DSGNLM_LIBRARY") or LIB_PATH


def load(path: str | None = None):
    """Load the compiled library.  Raises if it has not been built: there is no
    fallback implementation."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    default = path is None
    path = path or default_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -m paper_1901_06110_gb300.build)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if default:
        _lib = lib
    return lib
