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
