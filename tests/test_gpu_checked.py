"""The checked build (-DDSGNLM_CHECKED, lib/libdsgnlm_checked.so).

Its index checks test the computed offsets of the gathers and scattered writes against
the sizes of the buffers they address (weight planes, phase-1 partial regions, the
adjoint's G planes and window partials). A failed check sets a bit of a device word
and skips the access. These tests run in child processes that load the checked
library:

- the self test of the check itself, which touches no buffer;
- the DSG-NLM and adjoint parity suites under the checked build: every test must pass
  against the oracle and leave the check word at 0 (tests/conftest.py checks it after
  each test).

No test makes an out-of-range access.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checked_lib():
    from paper_1901_06110_gb300 import build
    return build.build(checked=True)


def _env(lib):
    env = dict(os.environ)
    env["DSGNLM_LIBRARY"] = lib
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    return env


SELFTEST = r"""
from paper_1901_06110_gb300 import dsgnlm as D
assert D.dsgnlm_is_checked()
assert D.dsgnlm_check_word(clear=True) == 0
D.dsgnlm_check_selftest(5, 10)
D.dsgnlm_check_selftest(0, 1)
assert D.dsgnlm_check_word() == 0
D.dsgnlm_check_selftest(10, 10)
assert D.dsgnlm_check_word() == 0x80000000
D.dsgnlm_check_selftest(-1, 10)
assert D.dsgnlm_check_word(clear=True) == 0x80000000
assert D.dsgnlm_check_word() == 0
print("selftest ok")
"""


def test_checked_build_selftest(checked_lib):
    r = subprocess.run([sys.executable, "-c", SELFTEST], cwd=ROOT, env=_env(checked_lib), capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "selftest ok" in r.stdout


def test_normal_build_has_no_checks(gpu_lib):
    from paper_1901_06110_gb300 import dsgnlm as D
    if os.environ.get("DSGNLM_LIBRARY"):
        pytest.skip("running under another library")
    assert not D.dsgnlm_is_checked()
    assert D.dsgnlm_check_word() == 0


@pytest.mark.parametrize("suite", ["tests/test_gpu_dsgnlm.py", "tests/test_gpu_adjoint.py",
                                   "tests/test_gpu_batched.py"])
def test_parity_suites_under_the_checked_build(checked_lib, suite):
    if os.environ.get("DSGNLM_REQUIRE_CLEAN_CHECK"):
        pytest.skip("already under the checked build")
    env = _env(checked_lib)
    env["DSGNLM_REQUIRE_CLEAN_CHECK"] = "1"
    r = subprocess.run([sys.executable, "-m", "pytest", suite, "-m", "gpu", "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-30:])
    assert r.returncode == 0, tail
