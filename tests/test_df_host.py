"""The double-float helpers of the refinement residual (csrc/df.cuh), built for
the host with g++ and checked against IEEE FP64 arithmetic: the exact widening
conversions, the error-free two-sums, and the FP64 <-> (hi, lo) round trip.
No GPU needed."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1107_2461_gb300", "csrc")


def test_df_helpers_match_ieee_fp64(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path / "df_host_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I" + CSRC, os.path.join(HERE, "df_host_check.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0 and res.stdout.strip().endswith("ok"), res.stdout + res.stderr
