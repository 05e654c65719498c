"""The host thread pool of the batched differentiable-form calls (csrc/host_pool.h),
compiled into a small program with the host compiler and run without a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1901_06110_gb300", "csrc")
CUDA = "/usr/local/cuda"


def test_host_pool_runs_every_index_once(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = tmp_path / "host_pool_check"
    cmd = [gxx, "-std=c++17", "-O1", "-pthread", "-I", CSRC, "-I", os.path.join(CUDA, "include"),
           os.path.join(ROOT, "tests", "host_pool_check.cpp"), "-o", str(exe),
           "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
