"""Compile the CUDA sources of this package into _build/libfeasm.so (sm_103a).

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library with the CUDA runtime linked statically.  The library is
rebuilt only when a source or header is newer than it.
"""

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfeasm.so")
# debug build: every FE_IN_BOUNDS index check compiled in (-DFE_DEBUG)
LIB_DEBUG = os.path.join(BUILD, "debug", "libfeasm_debug.so")
# HBM calibration probes used by the benchmark only (not part of libfeasm)
PROBE_SRC = os.path.join(CSRC, "probe", "hbm_probe.cu")
LIB_PROBE = os.path.join(BUILD, "probe", "libfeprobe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(ROOT, "include", "feasm.h"), os.path.abspath(__file__)]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(lib):
        return lib
    out_dir = os.path.dirname(lib)
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    flags = [*NVCC_FLAGS, *extra_flags, *(["-DFE_DEBUG"] if debug else [])]
    objs = []
    cmds = []
    for src in sources():
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        objs.append(obj)
        cmds.append([nvcc, *ARCH, *flags, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            print(" ".join(cmd))
            print(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {cmd[-3]}")
        return r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 4)) as ex:
        list(ex.map(run, cmds))
    tmp = lib + f".tmp{os.getpid()}"
    run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread"])
    os.replace(tmp, lib)
    return lib


def build_probe(force: bool = False) -> str:
    """The benchmark's HBM probe library (one translation unit)."""
    deps = [PROBE_SRC, os.path.join(CSRC, "tma.cuh"), os.path.abspath(__file__)]
    if not force and os.path.exists(LIB_PROBE) and all(os.path.getmtime(d) <= os.path.getmtime(LIB_PROBE)
                                                       for d in deps):
        return LIB_PROBE
    os.makedirs(os.path.dirname(LIB_PROBE), exist_ok=True)
    tmp = LIB_PROBE + f".tmp{os.getpid()}"
    cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, "-shared", "-cudart", "static", PROBE_SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        print(" ".join(cmd))
        print(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed on the probe library")
    os.replace(tmp, LIB_PROBE)
    return LIB_PROBE


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
