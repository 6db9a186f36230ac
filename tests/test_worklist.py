"""CPU check of the DK-pass work split (csrc/worklist.h, the host code that
cuts the plane tasks of a pass into per-CTA segments): compiled with g++ and
run on single lattices (block-aligned split), uneven ensembles (contiguous
cost-weighted split) and the up-only split of the U(1) pass; and of the
doublet pass's (tile, z-chunk) items (csrc/su2_work.h)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_worklist_covers_every_task_once(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = tmp_path / "worklist_check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-Wall", "-I",
                    os.path.join(ROOT, "paper_2102_01031_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "worklist_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.strip().splitlines()
    assert lines and all(l.startswith("OK") for l in lines), r.stdout
    # the headline shape keeps its largest per-CTA cost within 2 % of the mean
    bal = {l.split()[1]: float(l.split()[-1]) for l in lines if " balance " in l}
    assert bal["fp32_256_by8_g152"] < 1.02
    su2 = [l for l in lines if " su2_items " in l]
    assert len(su2) == 5
