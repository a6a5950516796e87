"""Build the library in-tree: nvcc for sm_103a, one object per source compiled in parallel,
linked into paper_1805_06607_gb300/_build/libsbpmrab.so (CUDA runtime linked statically); with
bounds_check=True, a build with SBP_BOUNDS_CHECK defined (the gathers check the table indices
they follow) into _build_checked/, loaded when SBP_MRAB_LIBRARY names it."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsbpmrab.so")
SOURCES = ["sbp_batch_f64.cu", "sbp_batch_f32.cu", "sbp_rhs_f64.cu", "sbp_rhs_f32.cu", "sbp_kernels.cu", "sbp_adjoint.cu",
           "sbp_capi.cpp", "sbp_adjoint_capi.cpp", "sbp_setup.cpp", "sbp_noalloc.cu", "sbp3_setup.cpp",
           "sbp3_kernels.cu", "sbp3_capi.cpp", "sbp3c_kernels.cu", "sbp3c_capi.cpp", "sbp3c_setup.cpp", "sbp_probe.cu", "sbp_faults.cu", "sbp_chain.cpp",
           "sbp3c_pair.cpp"]
HEADERS = ["sbp_internal.h", "sbp_device.h", "sbp_dev.cuh", "sbp_system.h", "sbp_rhs_impl.cuh", "sbp_march_impl.cuh", "sbp_march_tma.cuh", "sbp_col_impl.cuh", "sbp_batch_impl.cuh", "sbp3_device.h", "sbp3c_device.h", "sbp3_penalty.cuh", "sbp_tune.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _paths(bounds_check):
    out = os.path.join(HERE, "_build_checked") if bounds_check else OUT_DIR
    return out, os.path.join(out, "libsbpmrab.so")


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "sbp_mrab.h"),
                                                                  os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, bounds_check: bool = False) -> str:
    out_dir, lib = _paths(bounds_check)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    # host code without floating-point contraction, so that its arithmetic (coordinates, donor
    # search, Adams-Bashforth weights) is the same on x86 and Arm hosts
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "-I", os.path.join(ROOT, "include"), "-I", CSRC] + (["-DSBP_BOUNDS_CHECK"] if bounds_check else [])
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(out_dir, src + ".o")
        objs.append(obj)
        cmd = [nvcc, *ARCH, *common, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd[1:1] = ["-Xptxas", "-v"] if verbose else []
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, pr in procs:
        out, _ = pr.communicate()
        if verbose or pr.returncode:
            sys.stderr.write(out.decode(errors="replace"))
        if pr.returncode:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    tmp = lib + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds_check="--bounds-check" in sys.argv))
