"""Build libtn.so in-tree for sm_103a (GB300) with nvcc.

Every translation unit is compiled in parallel, then linked into
paper_2008_06888_gb300/libtn.so.  Run: python -m paper_2008_06888_gb300.build
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtn.so")
SOURCES = ["kernels.cu", "gate_count_i32.cu", "gate_count_f32.cu", "noalloc.cu", "planner.cpp",
           "program.cpp", "api.cpp", "jit.cpp", "sampler.cpp"]
# headers the run-time compiled chain kernels include (embedded into jit.cpp)
JIT_HEADERS = [("kJitTnInternal", "tn_internal.h"), ("kJitChainDev", "chain_dev.cuh")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
          "-Xcompiler", "-pthread",
          "-I" + os.path.join(os.path.dirname(HERE), "include")]


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _compile(src, verbose_ptxas=False):
    obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + ARCH + CFLAGS + ["-I" + OUT_DIR]
    if verbose_ptxas and src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def _write_jit_headers():
    """jit_headers.inc: the texts of JIT_HEADERS as C++ raw string literals."""
    out = []
    for var, name in JIT_HEADERS:
        text = open(os.path.join(CSRC, name)).read()
        if ")TNJIT" in text:
            raise RuntimeError(f"{name} contains the raw-string delimiter")
        out.append(f'static const char {var}[] = R"TNJIT({text})TNJIT";\n')
    path = os.path.join(OUT_DIR, "jit_headers.inc")
    data = "".join(out)
    if not os.path.exists(path) or open(path).read() != data:
        with open(path, "w") as f:
            f.write(data)


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    for d in (CSRC, os.path.join(os.path.dirname(HERE), "include")):
        for f in os.listdir(d):
            if os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return False


def build(force=False, verbose_ptxas=False):
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    _write_jit_headers()
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        res = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES))
    objs = [o for o, _ in res]
    if verbose_ptxas:
        for _, log in res:
            if log.strip():
                print(log, file=sys.stderr)
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart", "-lnvrtc", "-ldl", "-Xcompiler", "-pthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
