"""The separable index map (axis_offset, the offset of an aligned row or
column in an operand's reduced form; Sec. 2.3, Alg. 2) checked on the host
against a brute-force definition, for random product groups and maps: the
native check in tests/native is compiled with the host compiler against the
library's internal header and run (no GPU)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def test_axis_offset_matches_brute_force(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA runtime headers")
    exe = str(tmp_path / "axis_offset_check")
    src = os.path.join(HERE, "native", "axis_offset_check.cpp")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I",
                    os.path.join(ROOT, "paper_2007_08056_gb300", "csrc"), "-I", inc, src, "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok ")
