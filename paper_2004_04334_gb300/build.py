"""Build libhp.so in-tree with nvcc for sm_103a (one -gencode, two translation
units compiled in parallel, then linked against the shared CUDA runtime)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
BUILDDIR = os.path.join(ROOT, "_build")
LIB = os.path.join(LIBDIR, "libhp.so")

SOURCES = ["hp_kernels.cu", "hp_runtime.cpp", "hp_serving.cpp", "hp_tuning.cpp", "hp_switch.cpp", "hp_cpu.cpp",
           "hp_noalloc.cu", "hp_hits.cu", "hp_transfer.cu"]
HEADERS = [os.path.join(CSRC, "hp_internal.h"), os.path.join(CSRC, "hp_runtime.h"),
           os.path.join(CSRC, "hp_cpu.h"), os.path.join(INCLUDE, "hp.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home:
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _nvcc() -> str:
    nvcc = shutil.which("nvcc") or os.path.join(_cuda_home(), "bin", "nvcc")
    if not os.path.exists(nvcc):
        raise RuntimeError("nvcc not found: libhp needs the CUDA toolkit to build")
    return nvcc


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libhp.so if any source or header is newer; return its path."""
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    if not force and not _stale(LIB, srcs + HEADERS + [__file__]):
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    os.makedirs(BUILDDIR, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    procs = []
    objs = []
    for s in srcs:
        obj = os.path.join(BUILDDIR, os.path.basename(s) + ".o")
        objs.append(obj)
        cmd = [nvcc] + common + ["-c", s, "-o", obj]
        if verbose and s.endswith(".cu"):
            cmd += ["-Xptxas", "-v"]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = False
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode:
            sys.stderr.write("command failed: " + " ".join(cmd) + "\n")
            failed = True
    if failed:
        raise RuntimeError("libhp build failed")
    libdir = os.path.join(_cuda_home(), "lib64")
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "shared", "-Xlinker", f"-rpath,{libdir}",
                                                          "-lpthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode:
        sys.stderr.write(r.stdout.decode(errors="replace"))
        raise RuntimeError("libhp link failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
