"""Build libhelm.so in-tree with nvcc for sm_103a (GB300).

Each CUDA translation unit is compiled in parallel, then linked into one
shared library with a C ABI (include/helm.h).  No CMake; a minute or less.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhelm.so")
SOURCES = ["helm_api.cu", "k_setup.cu", "k_factor.cu", "k_stage.cu", "k_iface.cu", "k_iface_sym.cu", "k_krylov.cu", "k_mgs.cu", "k_adjoint.cu", "k_tc.cu",
           "habc_host.cu", "k_habc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                   "--expt-relaxed-constexpr"] + list(extra)


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src, os.path.join(CSRC, "helm_internal.cuh"), os.path.join(CSRC, "helm_check.cuh"),
            os.path.join(INCLUDE, "helm.h")]
    return any(os.path.getmtime(d) > t for d in deps)


# variant "check": the bounds-checking build (every checked global access of the kernels
# tested against the live device ranges, see csrc/helm_check.cuh) as libhelm_check.so
VARIANTS = {"": [], "check": ["-DHELM_CHECK_BOUNDS"]}


def build(verbose: bool = False, extra=(), variant: str = "") -> str:
    vflags = VARIANTS[variant]
    bdir = BUILD + ("_" + variant if variant else "")
    lib = LIB if not variant else os.path.join(HERE, f"libhelm_{variant}.so")
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(bdir, s.replace(".cu", ".o"))
        objs.append(obj)
        if _stale(obj, src) or extra:
            jobs.append([cc, "-c", src, "-o", obj] + flags(list(extra) + vflags))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if jobs or not os.path.exists(lib):
        cmd = [cc, "-shared", "-o", lib] + objs + ARCH + ["-cudart=static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
