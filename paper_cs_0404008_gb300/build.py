"""In-tree build of libgfpdot.so for sm_103a (nvcc, no cmake), of the
host sweep library libgfpsweep.so (plain C, the host compiler) and of the
measurement library libgfppeaks.so (nvcc).

Each CUDA translation unit under ``csrc/`` is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3`` and linked into
``_build/libgfpdot.so`` beside this file; ``sweep/gfp_sweep.c`` becomes
``_build/libgfpsweep.so``.  A build is skipped when its library is newer than
every source and header it depends on.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgfpdot.so")
SWEEP_SRC = os.path.join(HERE, "sweep", "gfp_sweep.c")
SWEEP_LIB = os.path.join(OUT, "libgfpsweep.so")
PEAKS_SRC = os.path.join(HERE, "peaks", "gfp_peaks.cu")
PEAKS_LIB = os.path.join(OUT, "libgfppeaks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgfpdot")


def _cuda_home(nvcc: str) -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return (sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


SAN_OUT = os.path.join(OUT, "sanitize")
SAN_LIB = os.path.join(SAN_OUT, "libgfpdot.so")
SAN_FLAGS = ["-fsanitize=address", "-fsanitize=undefined", "-fno-omit-frame-pointer",
             "-fno-sanitize-recover=undefined"]


DEBUG_OUT = os.path.join(OUT, "debug")
DEBUG_LIB = os.path.join(DEBUG_OUT, "libgfpdot.so")


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          sanitize: bool = False, debug: bool = False) -> str:
    """Compile and link libgfpdot.so; returns its path.  With sanitize=True the
    host code is built with AddressSanitizer and UndefinedBehaviorSanitizer
    into a separate library (_build/sanitize/libgfpdot.so) for host-side test
    runs (load it with libasan preloaded); device code is unchanged.  With
    debug=True the kernels keep their device-side checks (GFP_DEVICE_CHECKS:
    inputs outside the contract set error bits that gfp_context_check
    reports) in _build/debug/libgfpdot.so."""
    if sanitize and debug:
        raise ValueError("one variant at a time")
    out_dir, lib = (SAN_OUT, SAN_LIB) if sanitize else (DEBUG_OUT, DEBUG_LIB) if debug else (OUT, LIB)
    if not force and os.path.exists(lib) and all(os.path.getmtime(d) <= os.path.getmtime(lib)
                                                 for d in _deps()):
        return lib
    nvcc = _nvcc()
    os.makedirs(out_dir, exist_ok=True)
    common = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", "-I", os.path.join(ROOT, "include"),
              "-I", CSRC]
    if sanitize:
        common += [a for f in SAN_FLAGS for a in ("-Xcompiler", f)]
    if debug:
        common += ["-DGFP_DEVICE_CHECKS"]
    if ptxas_info:
        common += ["-Xptxas", "-v"]

    def compile_one(src: str) -> str:
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        cmd = common + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose or ptxas_info:
            print(r.stderr, end="")
        return obj

    srcs = sources()
    with ThreadPoolExecutor(max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, srcs))
    cuda_lib = os.path.join(_cuda_home(nvcc), "lib64")
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", f"-rpath={cuda_lib}", "-lpthread"]
    if sanitize:
        cmd += [a for f in SAN_FLAGS for a in ("-Xcompiler", f)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_sweep(force: bool = False) -> str:
    """Compile libgfpsweep.so with the host C compiler (-O2, no -march, so the
    same source builds on x86-64 and Arm); returns its path."""
    deps = [SWEEP_SRC, os.path.join(ROOT, "include", "gfpsweep.h"), os.path.abspath(__file__)]
    if (not force and os.path.exists(SWEEP_LIB)
            and all(os.path.getmtime(d) <= os.path.getmtime(SWEEP_LIB) for d in deps)):
        return SWEEP_LIB
    os.makedirs(OUT, exist_ok=True)
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        raise RuntimeError("no host C compiler found to build libgfpsweep")
    tmp = SWEEP_LIB + f".{os.getpid()}.tmp"
    cmd = [cc, "-O2", "-std=c11", "-fPIC", "-shared", "-fvisibility=default", "-I",
           os.path.join(ROOT, "include"), "-o", tmp, SWEEP_SRC, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"host compiler failed for {SWEEP_SRC}:\n{r.stderr}")
    os.replace(tmp, SWEEP_LIB)
    return SWEEP_LIB


def build_peaks(force: bool = False) -> str:
    """Compile libgfppeaks.so (the measured ceilings of the rooflines); returns its path."""
    deps = [PEAKS_SRC, os.path.join(ROOT, "include", "gfppeaks.h"), os.path.abspath(__file__)]
    if (not force and os.path.exists(PEAKS_LIB)
            and all(os.path.getmtime(d) <= os.path.getmtime(PEAKS_LIB) for d in deps)):
        return PEAKS_LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    cuda_lib = os.path.join(_cuda_home(nvcc), "lib64")
    tmp = PEAKS_LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler",
           "-fvisibility=hidden", "-I", os.path.join(ROOT, "include"), "-shared", "-cudart",
           "shared", "-o", tmp, PEAKS_SRC, "-Xlinker", f"-rpath={cuda_lib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {PEAKS_SRC}:\n{r.stderr}")
    os.replace(tmp, PEAKS_LIB)
    return PEAKS_LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
    print(build_sweep(force="--force" in sys.argv))
    print(build_peaks(force="--force" in sys.argv))
