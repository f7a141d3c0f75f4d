"""Builds libfcns.so (sm_103a) in-tree with nvcc and g++, compiling the
translation units in parallel.  Also builds libfcns_hostcheck.so, a CPU
execution of the kernel phase functions used only by the CPU tests to check
index arithmetic."""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build", platform.machine())
LIB = os.path.join(HERE, "libfcns.so")
HOSTCHECK = os.path.join(HERE, "libfcns_hostcheck.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-diag-suppress", "20013", "-I", os.path.join(ROOT, "include")]
CXX_FLAGS = ["-std=gnu++17", "-O2", "-fPIC", "-I", os.path.join(ROOT, "include")]

CU_SOURCES = ["k_deriv.cu", "k_deriv_f32.cu", "k_deriv_f64.cu", "k_deriv_noalloc.cu", "ns_capi.cu", "k_nsz_float.cu", "k_nsz_double.cu", "k_nsz_float_direct.cu", "k_nsz_float_alt.cu",
              "k_nsz_double_direct.cu", "k_nsxy_float.cu", "k_nsxy_double.cu",
              "k_nsx_float.cu", "k_nsx_double.cu", "k_probe.cu", "k_noise.cu"]
CPP_SOURCES = ["capi.cpp", "host_tables.cpp"]


def _cuda_home() -> str:
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r


def _newer(target: str, sources) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(s) <= t for s in sources)


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "fcns.h"), __file__]


def build(verbose: bool = False, hostcheck: bool = True) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    deps = _deps()
    jobs = []
    objs = []
    for s in CU_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        objs.append(o)
        if not _newer(o, deps):
            jobs.append([nvcc, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, s), "-o", o])
    for s in CPP_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        objs.append(o)
        if not _newer(o, deps):
            jobs.append(["g++", *CXX_FLAGS, "-I", os.path.join(cuda, "include"), "-c", os.path.join(CSRC, s), "-o", o])
    hc_src = os.path.join(CSRC, "hostcheck.cu")
    hc_obj = os.path.join(BUILD, "hostcheck.o")
    if hostcheck and os.path.exists(hc_src) and not _newer(hc_obj, deps):
        jobs.append([nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
                     "-diag-suppress", "20013", "-x", "cu", "-c", hc_src, "-o", hc_obj])
    with cf.ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        for r in ex.map(_run, jobs):
            if verbose:
                print(r.stdout, r.stderr, file=sys.stderr)
    stamp = os.path.join(BUILD, "lib.stamp")
    if not _newer(LIB, objs) or not _newer(stamp, [LIB]) or open(stamp).read() != platform.machine():
        _run(["g++", "-shared", "-o", LIB, *objs, "-L", os.path.join(cuda, "lib64"),
              "-Wl,-rpath," + os.path.join(cuda, "lib64"), "-lcudart"])
        with open(stamp, "w") as fh:
            fh.write(platform.machine())
    if hostcheck and os.path.exists(hc_obj) and not _newer(HOSTCHECK, [hc_obj]):
        _run(["g++", "-shared", "-o", HOSTCHECK, hc_obj, os.path.join(BUILD, "host_tables.cpp.o"),
              "-L", os.path.join(cuda, "lib64"), "-Wl,-rpath," + os.path.join(cuda, "lib64"), "-lcudart"])
    return LIB


def build_hostcheck_asan() -> str:
    """The host-check library built with AddressSanitizer and guard bands
    between the simulation's workspace arrays (for the CPU memory-safety
    test; load it into a process that preloads libasan).  Returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    cuda = _cuda_home()
    out = os.path.join(BUILD, "libfcns_hostcheck_asan.so")
    if _newer(out, _deps()):
        return out
    san = ["-fsanitize=address", "-fno-omit-frame-pointer"]
    hc_obj = os.path.join(BUILD, "hostcheck_asan.o")
    ht_obj = os.path.join(BUILD, "host_tables_asan.o")
    jobs = [[os.path.join(cuda, "bin", "nvcc"), "-std=c++17", "-O1", "--expt-relaxed-constexpr", "-DFC_LAYOUT_GUARD=256",
             "-Xcompiler", ",".join(["-fPIC"] + san), "-diag-suppress", "20013", "-x", "cu", "-c",
             os.path.join(CSRC, "hostcheck.cu"), "-o", hc_obj],
            ["g++", "-std=gnu++17", "-O1", "-fPIC", *san, "-I", os.path.join(ROOT, "include"), "-I",
             os.path.join(cuda, "include"), "-c", os.path.join(CSRC, "host_tables.cpp"), "-o", ht_obj]]
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        list(ex.map(_run, jobs))
    _run(["g++", "-shared", *san, "-o", out, hc_obj, ht_obj, "-L", os.path.join(cuda, "lib64"),
          "-Wl,-rpath," + os.path.join(cuda, "lib64"), "-lcudart"])
    return out


if __name__ == "__main__":
    print(build(verbose=True))
