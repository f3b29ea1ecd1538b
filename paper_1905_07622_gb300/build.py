"""Build the CUDA library libheatgb.so in-tree (nvcc, sm_103a only).

Each translation unit under csrc/ is compiled in parallel, then linked into
paper_1905_07622_gb300/lib/libheatgb.so. Objects go to _build/ (git-ignored).
build(checked=True) makes lib/libheatgb_check.so instead: the same sources
with HEAT_CHECK defined, whose kernels count out-of-range node and element
indices (heat_check_violations) instead of accessing them.
"""
from __future__ import annotations

import os
import platform
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build", platform.machine() or "host")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libheatgb.so")
LIB_CHECK = os.path.join(LIBDIR, "libheatgb_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libheatgb.so")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, extra_flags=None, checked: bool = False) -> str:
    """Compile every .cu under csrc/ for sm_103a and link libheatgb.so
    (libheatgb_check.so with the index checks when checked)."""
    bdir = BUILD + ("_check" if checked else "")
    lib = LIB_CHECK if checked else LIB
    os.makedirs(bdir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()
    hdrs = headers()
    extra = list(extra_flags or []) + (["-DHEAT_CHECK"] if checked else [])

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        if force or _stale(obj, [src] + hdrs):
            cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            if verbose and r.stderr.strip():
                print(r.stderr, flush=True)
        return obj

    srcs = sources()
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, srcs))
    stamp = os.path.join(LIBDIR, ".machine" + ("_check" if checked else ""))
    same_machine = os.path.exists(stamp) and open(stamp).read().strip() == platform.machine()
    if force or not same_machine or _stale(lib, objs):
        cmd = [cc, *ARCH, "-shared", "-o", lib, *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        with open(stamp, "w") as fh:
            fh.write(platform.machine())
    return lib


if __name__ == "__main__":
    import sys

    print(build(verbose=True, force="--force" in sys.argv))
