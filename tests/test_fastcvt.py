"""The integer-operation conversions between binary64 and binary32 that the
MIXED refinement's FP32 steps use (csrc/fastcvt.h), compiled for the host
with g++ (the header is plain C++ for host and device) and compared bit for
bit with the C++ conversions, which round to nearest even: 2M random values
over the binary32 normal range, the same values moved to exact ties, the
binary32 -> binary64 direction, and the documented edges (signed zero below
2^-126, signed infinity above the binary32 range, FLT_MAX kept)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fastcvt_check.cpp")
INC = os.path.join(os.path.dirname(HERE), "paper_2303_04992_gb300", "csrc")


def test_fastcvt_matches_host_conversions(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path / "fastcvt_check")
    subprocess.run(["g++", "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror", "-I", INC, SRC, "-o", exe],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=300).stdout
    got = {k: int(v) for k, v in (line.split() for line in out.splitlines())}
    assert got["n"] == 2000000
    for k in ("random", "ties", "back", "small", "big"):
        assert got[k] == 0, got
