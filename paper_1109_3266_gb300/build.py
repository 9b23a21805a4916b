"""Build the dose engine's CUDA library (sm_103a) in-tree:
paper_1109_3266_gb300/_build/libctd.so.

Every translation unit is compiled in parallel with
    nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo -O3
the transport kernels with --use_fast_math (hardware reciprocal, square root,
logarithm and sincos, contracted multiply-adds; binary64 is unaffected), the
other kernels with --fmad=false, and host code with -ffp-contract=off, so that
the host-built tables do not depend on the host compiler's FMA contraction.
"""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libctd.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["ctd_capi.cu", "ctd_forms.cu", "ctd_tune.cu", "ctd_transport.cu", "ctd_stats.cu", "ctd_physics.cpp",
           "ctd_noalloc.cu", "ctd_probe.cu", "ctd_fluence.cu"]
HEADERS = ["ctd_internal.h", "ctd_host.h", "ctd_device.cuh"]
FAST_MATH = {"ctd_transport.cu"}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
HOST_FLAGS = "-fPIC,-ffp-contract=off,-fno-fast-math,-O2"


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(SRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "ctd.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra) -> str:
    obj = os.path.join(OUT, os.path.basename(src) + ".o")
    fp = ["--use_fast_math"] if src in FAST_MATH else ["--fmad=false"]
    cmd = [nvcc(), *ARCH, "-lineinfo", "-O3", *fp, "-std=c++17", "-I", INCLUDE,
           "-Xcompiler", HOST_FLAGS, "-c", os.path.join(SRC, src), "-o", obj, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile the library if any source changed; return its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
