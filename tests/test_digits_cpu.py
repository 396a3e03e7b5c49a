"""The digit decomposition of the tensor-core phases, checked on the host.

Compiles tests/digits_check.cpp (g++, CUDA headers for the FP8 conversion)
against paper_2203_05665_gb300/csrc/h2_digits.hpp and runs it: digits within
[-16, 16], exact reconstruction, exact E4M3 encoding of every digit, and the
truncation bound of the kept digit pairs, on boundary values and 2e6 random
pairs per digit count.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"


def test_digit_split_and_truncation_bound(tmp_path):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    exe = tmp_path / "digits_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CUDA_INC,
                    "-I", os.path.join(ROOT, "paper_2203_05665_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "digits_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
