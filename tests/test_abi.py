"""The C ABI library builds, loads and exports every function include/dsgnlm.h
declares; argument checks that run before any CUDA call.  CPU only."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared_functions():
    names = set()
    for hdr in HEADERS:
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b([a-z][a-z0-9_]+)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name.startswith(("dsgnlm_", "lpnp_")):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1901_06110_gb300 import _abi, build
    build.build()
    return _abi.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_1901_06110_gb300 import _abi
    declared = _declared_functions()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    # the binding declares exactly the header's functions
    assert declared == set(_abi.SIGNATURES), declared ^ set(_abi.SIGNATURES)


def test_library_is_sm_103a_only():
    from paper_1901_06110_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_status_strings(lib):
    for s in range(9):
        assert lib.dsgnlm_strerror(s)
    assert lib.dsgnlm_strerror(0) == b"ok"


def test_host_side_argument_checks(lib):
    from paper_1901_06110_gb300 import _abi
    h = ctypes.c_void_p()
    assert lib.dsgnlm_create(None, None, 0) == _abi.EINVAL
    assert lib.dsgnlm_create(ctypes.byref(h), None, 7) == _abi.EINVAL
    assert lib.dsgnlm_create(ctypes.byref(h), None, _abi.F16) == _abi.OK
    try:
        fake = ctypes.c_void_p(0x10000)  # never dereferenced: rejected before any CUDA call
        assert lib.dsgnlm_build(h, None, 8, 8, 1, 1, 0.1) == _abi.EINVAL
        assert lib.dsgnlm_build(h, fake, 0, 8, 1, 1, 0.1) == _abi.EINVAL
        assert lib.dsgnlm_build(h, fake, 8, 8, 15, 1, 0.1) == _abi.EINVAL
        assert lib.dsgnlm_build(h, fake, 8, 8, 1, 25, 0.1) == _abi.EINVAL
        assert lib.dsgnlm_build(h, fake, 8, 8, 1, 1, 0.0) == _abi.EINVAL
        assert lib.dsgnlm_build(h, ctypes.c_void_p(0x10004), 8, 8, 1, 1, 0.1) == _abi.EINVAL
        assert lib.dsgnlm_balance(h, 1e-6, 10, None, None) == _abi.NOT_BUILT
        assert lib.dsgnlm_apply(h, fake, ctypes.c_void_p(0x20000)) == _abi.NOT_BUILT
        assert lib.dsgnlm_apply(h, fake, fake) == _abi.EINVAL
        assert lib.dsgnlm_num_offsets(h) == 0
        p = _abi.LpnpProblem()
        assert lib.lpnp_solve(None, 1.0, 1) == _abi.EINVAL
        assert lib.lpnp_solve(ctypes.byref(p), 1.0, 1) == _abi.EINVAL
        t = ctypes.c_void_p()
        assert lib.lpnp_tape_create(ctypes.byref(t)) == _abi.OK
        try:
            tapes = (ctypes.c_void_p * 2)(t.value, t.value)
            dens = (ctypes.c_void_p * 2)(h.value, h.value)
            ptrs = (ctypes.c_void_p * 2)(0x10000, 0x20000)
            args = (8, 8, 1, 1, 0.1, 2, 1.0, 1.0, 2, 1.0, 1, ptrs)
            assert lib.lpnp_unrolled_forward_batched(tapes, dens, 0, ptrs, ptrs, *args) == _abi.EINVAL
            assert lib.lpnp_unrolled_forward_batched(tapes, dens, 2, ptrs, ptrs, *args) == _abi.EINVAL  # repeats
            assert lib.lpnp_unrolled_forward_batched(None, dens, 1, ptrs, ptrs, *args) == _abi.EINVAL
            assert lib.lpnp_backward_batched(tapes, 2, ptrs, ptrs, ptrs, None, None) == _abi.EINVAL  # repeats
            assert lib.lpnp_backward_batched(tapes, 1, ptrs, ptrs, ptrs, None, None) == _abi.EINVAL  # not recorded
            assert lib.lpnp_backward(t, fake, fake, fake, None, None) == _abi.EINVAL
        finally:
            lib.lpnp_tape_destroy(t)
    finally:
        lib.dsgnlm_destroy(h)
    assert lib.dsgnlm_launch_count() == 0


def test_binding_raises_without_library(tmp_path):
    from paper_1901_06110_gb300 import _abi
    with pytest.raises(RuntimeError, match="missing"):
        _abi.load(str(tmp_path / "nope.so"))
