"""Build of the in-tree CUDA libraries ``liblbfreeze.so`` (the LB step) and ``libcno.so`` (the learned surrogate) for sm_103a with nvcc."""
from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "liblbfreeze.so")
CNO_LIB = os.path.join(PKG, "libcno.so")

# (library, sources, headers it depends on)
TARGETS = [
    (LIB, ["lb_api.cu"], ["lb_kernels.cuh", "lbfreeze.h"]),
    (CNO_LIB, ["cno_api.cu"], ["cno_kernels.cuh", "cno.h"]),
]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the CUDA libraries")


def _dep_path(name: str) -> str:
    return os.path.join(INCLUDE if name.endswith(".h") else CSRC, name)


def _stale(lib: str, sources, headers) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in sources] + [_dep_path(h) for h in headers] + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the libraries for sm_103a if missing or older than their sources
    (the two nvcc processes run in parallel).  Returns the path of liblbfreeze.so."""
    jobs = []
    for lib, sources, headers in TARGETS:
        if not force and not _stale(lib, sources, headers):
            continue
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [nvcc()] + ARCH + NVCC_FLAGS + ["-I", INCLUDE, "-o", tmp] + [os.path.join(CSRC, s) for s in sources]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((lib, tmp, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
    errors = []
    for lib, tmp, cmd, proc in jobs:
        out, err = proc.communicate()
        if proc.returncode != 0:
            errors.append("nvcc failed:\n" + " ".join(cmd) + "\n" + out + err)
            continue
        if verbose:
            print(out + err)
        os.replace(tmp, lib)
    if errors:
        raise RuntimeError("\n".join(errors))
    return LIB
