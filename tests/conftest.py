import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    # GPU tests cannot run without a device; skip them instead of failing.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library, built in-tree if needed (GPU tests only)."""
    from paper_1901_06110_gb300 import _abi, build
    build.build()
    return _abi.load()


@pytest.fixture(autouse=True)
def _clean_check_word(request):
    """Under the checked build (the parity tests rerun by test_gpu_checked.py, with
    DSGNLM_REQUIRE_CLEAN_CHECK set), every GPU test must leave the index-check word at 0:
    no gather or scattered write of the library left its buffer."""
    yield
    if os.environ.get("DSGNLM_REQUIRE_CLEAN_CHECK") and "gpu" in request.keywords:
        from paper_1901_06110_gb300 import dsgnlm as D
        word = D.dsgnlm_check_word(clear=True)
        assert word == 0, f"checked build: index-check word {word:#x} after {request.node.nodeid}"
