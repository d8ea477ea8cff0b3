"""In-tree build of liblsms.so for sm_103a (nvcc, one -gencode, translation units in parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblsms.so")
SOURCES = ["abi.cu", "kernels_f64.cu", "mixed.cu", "contour_tc.cu", "translate_tc.cu", "gmres.cu", "batch.cu",
           "host_setup.cpp", "inclusion.cpp", "fmm.cu"]
# The benchmark's FMA-pipe probe: a library of its own, outside the lsms ABI.
PROBE_SRC = os.path.join(CSRC, "probe", "fma_probe.cu")
PROBE_LIB = os.path.join(OUT_DIR, "libfmaprobe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblsms")
    return nvcc


def build_probe(nvcc: str) -> str:
    """libfmaprobe.so from csrc/probe/fma_probe.cu (rebuilt when the source is newer)."""
    if os.path.exists(PROBE_LIB) and os.path.getmtime(PROBE_LIB) >= os.path.getmtime(PROBE_SRC):
        return PROBE_LIB
    tmp = PROBE_LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-shared", "-cudart", "static",
           PROBE_SRC, "-o", tmp]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on fma_probe.cu:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def build(verbose: bool = False, jobs: int | None = None) -> str:
    """Compile every source and link liblsms.so (and the benchmark's libfmaprobe.so); returns the
    library's path.  Rebuilds only when a source or header is newer than the library."""
    os.makedirs(OUT_DIR, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if os.path.isfile(os.path.join(CSRC, f))]
    deps.append(os.path.join(ROOT, "include", "lsms.h"))
    nvcc = _nvcc()
    with cf.ThreadPoolExecutor(max_workers=1) as ex_probe:
        probe = ex_probe.submit(build_probe, nvcc)
        if not (os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps)):
            _build_lib(nvcc, verbose, jobs)
        probe.result()
    return LIB


def _build_lib(nvcc: str, verbose: bool, jobs: int | None) -> None:

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT_DIR, src + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        if verbose and (res.stdout or res.stderr):
            print(res.stdout, res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=jobs or len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-L" + cuda_lib,
           "-Xlinker", "-rpath=" + cuda_lib]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)


if __name__ == "__main__":
    print(build(verbose=True))
