"""Register-chain fold on the host: the folded table gates of every chain
evaluate exactly like the original gate lists (tests/host/fold_check.cpp,
compiled here with g++ against the planner and program builder)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2008_06888_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime_api.h")):
            return os.path.join(d, "include")
    return None


@pytest.mark.timeout(300)
def test_folded_tables_equal_gate_lists(tmp_path):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("g++ or CUDA headers missing")
    exe = str(tmp_path / "fold_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-I", CSRC, "-I", inc,
                    os.path.join(ROOT, "tests", "host", "fold_check.cpp"),
                    os.path.join(CSRC, "planner.cpp"), os.path.join(CSRC, "program.cpp"),
                    "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stdout + r.stderr
    last = r.stdout.strip().splitlines()[-1].split()
    # "chains C orig gates G table gates T mismatches 0"
    chains, orig, folded = int(last[1]), int(last[4]), int(last[7])
    assert chains > 100 and folded < orig and last[-1] == "0"
