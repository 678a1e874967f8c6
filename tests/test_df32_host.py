"""Host checks of the exact FP64 <-> FP32-pair conversions used by the compensated-FP32 precision."""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_df32_conversions_roundtrip(tmp_path):
    exe = tmp_path / "df32_roundtrip"
    src = os.path.join(HERE, "df32_roundtrip.cpp")
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", src, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok")


def test_df_tanh_against_long_double(tmp_path):
    """tanh and 1 - tanh^2 in compensated FP32 pairs (dfmath.h, the compensated-FP32 form's chain
    maps): relative error of tanh and absolute error of 1 - tanh^2 below 2^-45 over 2e6 arguments
    from 1e-30 to 40 of both signs, the branch edges (1/4, 19.1), zero, subnormals, infinities and
    NaN, against long double tanhl."""
    exe = tmp_path / "df_tanh_check"
    src = os.path.join(HERE, "df_tanh_check.cpp")
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", src, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok")
