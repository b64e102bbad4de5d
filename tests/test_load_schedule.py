"""Host logic of Newton's load schedule (equal steps, halved increments after a failed level,
regrowth, cut limits): compiles tests/cpp/load_schedule_test.cpp against the library's
internal header with the host compiler and runs it (no GPU)."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2601_03086_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


def test_load_schedule(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "load_schedule_test")
    src = os.path.join(ROOT, "tests", "cpp", "load_schedule_test.cpp")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", CUDA_INC, src, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
