"""Compiles the CUDA library ``_build/libdisco.so`` for sm_103a with nvcc.

Translation units are compiled in parallel and linked into one shared library
with a plain C ABI (``include/disco.h``). Rebuilds only when a source is newer
than the library.

With the environment variable ``DISCO_BOUNDS_CHECK=1`` the library is built
with device-side index checks in the half-pass kernels (an index outside its
array sets a status bit and the access is skipped; the host reports
DISCO_ERR_INTERNAL) into ``_build_bc/``, and the binding loads that one.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BOUNDS_CHECK = os.environ.get("DISCO_BOUNDS_CHECK", "0") not in ("", "0")
OUT_DIR = os.path.join(HERE, "_build_bc" if BOUNDS_CHECK else "_build")
LIB = os.path.join(OUT_DIR, "libdisco.so")
SOURCES = ["disco.cu", "kernels.cu", "adjoint.cu", "qn.cu", "store.cu", "host_build.cpp", "noalloc.cu"]
HEADERS = ["plan.h", "kernels.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    deps.append(os.path.join(HERE, "..", "include", "disco.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3", "--expt-relaxed-constexpr"] + ARCH
    if BOUNDS_CHECK:
        common.append("-DDISCO_BOUNDS_CHECK")
    procs, objs = [], []
    for s in SOURCES:
        obj = os.path.join(OUT_DIR, os.path.splitext(s)[0] + ".o")
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, s), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), cmd))
        objs.append(obj)
    for p, cmd in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(cmd) + "\n" + out.decode(errors="replace"))
        if verbose and out:
            print(out.decode(errors="replace"))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, "-shared"] + ARCH + ["-o", tmp] + objs + ["-lpthread"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + " ".join(cmd) + "\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
