"""Host-side checks of the chain program, compiled here with g++ against the
planner and program builder (no GPU):

- tests/host/fold_check.cpp: the folded table gates of every register chain
  evaluate exactly like the original gate lists;
- tests/host/tile_check.cpp: the coalesced tile copies of compiled chains put
  every element where its owning thread reads it, without bank conflicts;
- tests/host/sample_check.cpp: the ground-state sampler with brute-force counts;
- tests/host/perm_check.cpp: the index map of the tiled q = 2 transpose."""
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


def _build_check(tmp_path, name, extra_src=(), libs=()):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("g++ or CUDA headers missing")
    exe = str(tmp_path / name)
    cmd = ["g++", "-O2", "-std=c++17", "-pthread", "-I", CSRC, "-I", inc,
           os.path.join(ROOT, "tests", "host", name + ".cpp"),
           os.path.join(CSRC, "planner.cpp"), os.path.join(CSRC, "program.cpp")]
    cmd += [os.path.join(CSRC, s) for s in extra_src] + ["-o", exe] + list(libs)
    subprocess.run(cmd, check=True)
    return exe


@pytest.mark.timeout(300)
def test_folded_tables_equal_gate_lists(tmp_path):
    exe = _build_check(tmp_path, "fold_check")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stdout + r.stderr
    last = r.stdout.strip().splitlines()[-1].split()
    # "chains C orig gates G table gates T mismatches 0"
    chains, orig, folded = int(last[1]), int(last[4]), int(last[7])
    assert chains > 100 and folded < orig and last[-1] == "0"


@pytest.mark.timeout(300)
def test_tile_copies_of_compiled_chains(tmp_path):
    from paper_2008_06888_gb300 import build
    build.build()   # writes the embedded header texts jit.cpp includes
    cuda_lib = os.path.join(os.path.dirname(_cuda_include() or "/usr/local/cuda/include"), "lib64")
    exe = _build_check(tmp_path, "tile_check", extra_src=("jit.cpp",),
                       libs=("-I" + build.OUT_DIR, "-L" + cuda_lib, "-lnvrtc", "-lcudart", "-ldl"))
    env = dict(os.environ, LD_LIBRARY_PATH=cuda_lib + ":" + os.environ.get("LD_LIBRARY_PATH", ""))
    # default slot layout (at most one low register leg) and the two-leg form
    for low_max in ("1", "2"):
        env["TN_JIT_LOW_MAX"] = low_max
        r = subprocess.run([exe], capture_output=True, text=True, timeout=240, env=env)
        assert r.returncode == 0, r.stdout + r.stderr
        assert "wrong 0 bank_conflicts 0" in r.stdout and "compiled 6 failed 0" in r.stdout


@pytest.mark.timeout(300)
def test_ground_state_sampler_with_brute_force_counts(tmp_path):
    """tests/host/sample_check.cpp: the conditional-count sampler (Sec. III) draws
    only ground states, uniformly, independent of its batch size."""
    if shutil.which("g++") is None:
        pytest.skip("g++ missing")
    exe = str(tmp_path / "sample_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC,
                    os.path.join(ROOT, "tests", "host", "sample_check.cpp"),
                    os.path.join(CSRC, "sampler.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().splitlines()[-1].endswith("bad 0")


@pytest.mark.timeout(300)
def test_tiled_transpose_map(tmp_path):
    """tests/host/perm_check.cpp: the q = 2 tiled transpose (k_permute2) writes every
    output element once from the element the permutation defines, with coalesced
    32-element warp accesses and no shared-memory bank conflicts."""
    if shutil.which("g++") is None:
        pytest.skip("g++ missing")
    exe = str(tmp_path / "perm_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC,
                    os.path.join(ROOT, "tests", "host", "perm_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "wrong 0 bank_conflicts 0 uncoalesced 0" in r.stdout
