"""Build libldgmg.so (the C-ABI library) in-tree for sm_103a.

Translation units are compiled in parallel (one nvcc/g++ process each) and
linked with nvcc.  The result lands next to this file; objects go to _build/.
Usage: python -m paper_2412_12506_gb300.build
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libldgmg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _run_parallel(cmds):
    procs = [(c, subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)) for c in cmds]
    failed = []
    for c, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((c, text))
        elif text.strip() and os.environ.get("LDGMG_BUILD_VERBOSE"):
            sys.stderr.write(text)
    if failed:
        msg = "\n\n".join(" ".join(c) + "\n" + t for c, t in failed)
        raise RuntimeError("libldgmg build failed:\n" + msg)


def build(verbose: bool = False, extra_nvcc=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common_inc = ["-I", INCLUDE, "-I", CSRC]
    objs, cmds = [], []
    for src in sorted(os.listdir(CSRC)):
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        if src.endswith(".cu"):
            cmds.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                         "--expt-relaxed-constexpr", *common_inc, *extra_nvcc, "-c", path, "-o", obj])
        elif src.endswith(".cpp"):
            cuda_inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
            cmds.append(["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", *common_inc, "-I", cuda_inc,
                         "-c", path, "-o", obj])
        else:
            continue
        objs.append(obj)
    if verbose:
        for c in cmds:
            print(" ".join(c))
    _run_parallel(cmds)
    tmp = LIB + ".tmp"
    link = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs,
            "-lcusolver", "-lcublas", "-lpthread"]
    _run_parallel([link])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
