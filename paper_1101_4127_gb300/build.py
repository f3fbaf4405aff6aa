"""Build libcrash.so (the C ABI of include/crash.h) for sm_103a with nvcc.

Translation units are compiled in parallel; the FP64 transport unit is built
with -fmad=false so that it reproduces the FP64 step specification bit for
bit.  Output goes to paper_1101_4127_gb300/_build/ (git-ignored)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "libcrash.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# (source, extra flags)
UNITS = [
    ("crash_api.cu", []),
    ("k_fp64.cu", ["-fmad=false"]),
    ("k_chem.cu", []),
    ("k_mixed.cu", ["-fmad=false"]),   # explicit fmaf only: every launch shape rounds alike
    ("k_noalloc.cu", []),
]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "crash.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= _deps():
        return SO
    # host code: no FP contraction (the host-side tables must match the FP64
    # specification on every host architecture, aarch64 included)
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "-Xptxas", "-v" if verbose else "-O3",
              "-I", os.path.join(ROOT, "include")] + ARCH

    def compile_one(u):
        src, extra = u
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + common + extra
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        res = list(ex.map(compile_one, UNITS))
    if verbose:
        for _, log in res:
            sys.stderr.write(log)
    tmp = SO + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-shared", "-o", tmp] + [o for o, _ in res] + ARCH + ["-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr)
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
