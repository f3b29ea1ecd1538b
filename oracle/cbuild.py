"""Build the oracle's plain C solvers (oracle/cpcg.c) into a shared library
(test infrastructure and the timed CPU baseline only).

gcc with OpenMP, no machine-specific flags, into _build/oracle/<machine>/
(git-ignored); rebuilt when the source is newer than the library.
"""
from __future__ import annotations

import os
import platform
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "cpcg.c")
LIB = os.path.join(ROOT, "_build", "oracle", platform.machine() or "host", "liboracle_cpu.so")


def build(verbose: bool = False) -> str:
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = os.environ.get("CC") or shutil.which("gcc") or shutil.which("cc")
    if not cc:
        raise RuntimeError("no C compiler for the oracle's C solvers")
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    cmd = [cc, "-O2", "-fopenmp", "-fPIC", "-shared", "-o", LIB, SRC, "-lm"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"oracle C build failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
