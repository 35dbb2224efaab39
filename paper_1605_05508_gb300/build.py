"""Build step of libkf: compiles csrc/*.cu for sm_103a (GB300) with nvcc into
paper_1605_05508_gb300/_build/libkf.so.  Translation units compile in
parallel; the library links against the CUDA runtime only.  Also links the
native serving driver (serve_driver.c) against it: _build/kf_serve_driver."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC_DIR = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libkf.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: the kernels write every fused multiply-add explicitly; without
# implicit contraction each kernel form rounds a track identically
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-DNDEBUG", "-fmad=false",
              "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc() -> str:
    cand = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cand, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def _stale(srcs, lib) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = srcs + glob.glob(os.path.join(SRC_DIR, "*.cuh")) + glob.glob(os.path.join(SRC_DIR, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.join(HERE, "serve_driver.c")]
    if not os.path.exists(os.path.join(OUT_DIR, "kf_serve_driver")):
        return True
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    srcs = sorted(glob.glob(os.path.join(SRC_DIR, "*.cu")))
    if not force and not _stale(srcs, LIB):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    procs, objs = [], []
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    for s in srcs:
        o = os.path.join(OUT_DIR, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", s, "-o", o]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for s, p in procs:
        out, _ = p.communicate()
        if out and (verbose or ptxas_info or p.returncode):
            print(out, file=sys.stderr)
        if p.returncode:
            failed.append(s)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], check=True)
    os.replace(tmp, LIB)
    build_serve_driver(verbose)
    return LIB


DRIVER_SRC = os.path.join(HERE, "serve_driver.c")
DRIVER = os.path.join(OUT_DIR, "kf_serve_driver")


def build_serve_driver(verbose: bool = False) -> str:
    """The native serving driver (serve_driver.c) linked against libkf."""
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc())), "lib64")
    cmd = ["gcc", "-O2", "-std=gnu11", "-I", INCLUDE, DRIVER_SRC, "-o", DRIVER + f".tmp{os.getpid()}",
           "-L", OUT_DIR, "-lkf", f"-Wl,-rpath,{OUT_DIR}", f"-Wl,-rpath,{cuda_lib}", "-lpthread", "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(DRIVER + f".tmp{os.getpid()}", DRIVER)
    return DRIVER


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv)
