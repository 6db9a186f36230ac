"""CPU check of the autotuner's on-disk cache (paper_2102_01031_gb300/csrc/tune_cache.h,
used by cl_set_tune_cache)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tune_cache_file(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = tmp_path / "tune_cache_check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-Wall", "-I",
                    os.path.join(ROOT, "paper_2102_01031_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "tune_cache_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe), str(tmp_path)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.strip().splitlines()
    assert len(lines) == 5 and all(l.startswith("OK") for l in lines), r.stdout
