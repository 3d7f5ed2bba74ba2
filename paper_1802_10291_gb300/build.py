"""Build the CUDA library ``_build/libmci.so`` in-tree for sm_103a (GB300).

Translation units compile in parallel with nvcc, then link into one shared
library exporting the C ABI of ``include/mci.h``.  Run as a script or call
:func:`build`.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmci.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++20", "-rdc=true", "-Xcompiler", "-fPIC", "-Xcompiler",
              "-O2", "--expt-relaxed-constexpr", "-DNDEBUG", f"-I{os.path.join(ROOT, 'include')}"]
# host plan code is plain C++ (g++); kernels and the device-side scheduler are CUDA with
# relocatable device code, because the scheduler launches the size-class kernels.
HOST_UNITS = ["mci_host.cpp", "mci2d_host.cpp"]
CUDA_UNITS = ["mci_fast.cu", "mci_mirror.cu", "mci_sched.cu", "mci_noalloc.cu", "mci_gemm.cu", "mci_error.cu", "mci_corrector.cu", "mci2d.cu", "k_lookup.cu", "k_a.cu", "k_b.cu", "k_c.cu", "k_d.cu", "k_e.cu"]
UNITS = HOST_UNITS + CUDA_UNITS


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def cuda_home() -> str:
    cc = nvcc()
    if os.path.sep in cc:
        return os.path.dirname(os.path.dirname(os.path.realpath(cc)))
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _sources_newer(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not force and not _sources_newer(LIB):
        return LIB
    cc = nvcc()

    def compile_unit(u: str) -> str:
        obj = os.path.join(BUILD, os.path.splitext(u)[0] + ".o")
        if u in HOST_UNITS:
            cmd = [os.environ.get("CXX", "g++"), "-std=c++17", "-O2", "-fPIC",
                   f"-I{os.path.join(cuda_home(), 'include')}", f"-I{os.path.join(ROOT, 'include')}",
                   "-c", os.path.join(CSRC, u), "-o", obj]
        else:
            cmd = [cc, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, u), "-o", obj]
            if ptxas_verbose:
                cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {u}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-rdc=true", "-o", tmp, *objs, "-lcudadevrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv))
