"""Build libqss.so (host runtime, CUDA driver API) and qss_aux.cubin (sm_103a).

    python -m paper_2405_05974_b300.build_ext

Both products are written next to this file; the runtime finds the auxiliary
cubin beside itself.
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
REPO = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(REPO, "include")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
LIB = os.path.join(PKG, "libqss.so")
AUX = os.path.join(PKG, "qss_aux.cubin")
SOURCES = ["qss_driver.cpp", "qss_runtime.cpp", "qss_implicit.cpp", "qss_integrate.cpp", "qss_probe.cpp",
           "qss_serve.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


NOALLOC = "qss_noalloc.cu"   # the only CUDA-runtime translation unit (static cudart)


def build(force: bool = False, verbose: bool = False):
    srcs = [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    hdrs = [os.path.join(CSRC, "qss_internal.h"), os.path.join(CSRC, "qss_driver.h"), os.path.join(INCLUDE, "qss.h")]
    cu = os.path.join(CSRC, NOALLOC)
    obj = os.path.join(PKG, "qss_noalloc.o")
    if force or _newer(obj, [cu] + hdrs):
        cmd = ["nvcc", "-c", *ARCH, "-O3", "-Xcompiler", "-fPIC", "-std=c++17", "-I", INCLUDE, "-I", CSRC,
               "-o", obj + ".tmp.o", cu]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        os.replace(obj + ".tmp.o", obj)
    if force or _newer(LIB, srcs + hdrs + [obj]):
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-Wall", "-Wextra", "-Wno-unused-parameter",
               "-I", INCLUDE, "-I", CSRC, "-I", os.path.join(CUDA_HOME, "include"), "-o", LIB + ".tmp",
               *srcs, obj, "-L", os.path.join(CUDA_HOME, "lib64"), "-lcudart_static", "-lrt",
               "-lpthread", "-ldl"]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    aux_src = os.path.join(CSRC, "qss_aux.cu")
    aux_deps = [aux_src, os.path.join(CSRC, "qss_device.cuh"), os.path.join(CSRC, "qss_exp_table.inc")]
    if force or _newer(AUX, aux_deps):
        cmd = ["nvcc", "-cubin", *ARCH, "-O3", "-lineinfo", "-I", CSRC, "-o", AUX + ".tmp", aux_src]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        os.replace(AUX + ".tmp", AUX)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
