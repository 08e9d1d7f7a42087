"""Build the KLB CUDA library in-tree (``paper_2403_15768_gb300/_build/libklb.so``).

Plain nvcc for sm_103a, one translation unit per source compiled in
parallel, then one shared-library link.  No torch extension machinery: the
library exposes only the C ABI of ``include/klb.h``.  ``bounds=True``
builds the debug variant with index checks (``-DKLB_BOUNDS=1``) into
``_build_bounds/``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libklb.so")
SOURCES = ["klb_kernels_q19.cu", "klb_kernels_q9.cu", "klb_kernels.cu", "klb_geometry.cpp",
           "klb_api.cpp", "klb_static.cu", "klb_server.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the KLB library needs the CUDA toolkit")
    return path


def _inputs():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(ROOT, "include", "klb.h"))
    return [os.path.join(CSRC, s) for s in SOURCES] + hdrs + [__file__]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags=(), bounds: bool = False) -> str:
    build_dir = BUILD + "_bounds" if bounds else BUILD
    lib = os.path.join(build_dir, "libklb.so")
    if not force and up_to_date(lib):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    flags = [*extra_flags, *(["-DKLB_BOUNDS=1"] if bounds else [])]
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
              "-I", os.path.join(ROOT, "include"), "-I", CSRC, *ARCH, *flags]
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(build_dir, src.rsplit(".", 1)[0] + ".o")
        objs.append(obj)
        cmd = [nvcc(), *common, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if pr.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds="--bounds" in sys.argv))
