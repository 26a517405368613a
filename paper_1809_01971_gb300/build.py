"""Build libfc.so in-tree for sm_103a (nvcc for the CUDA sources, g++ for the host setup).

Translation units are compiled in parallel and linked with nvcc.  Output:
paper_1809_01971_gb300/libfc.so (git-ignored).  Run ``python -m paper_1809_01971_gb300.build``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libfc.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["api.cu", "k_fft.cu", "k_linalg.cu", "k_symeig.cu", "k_tensor.cu", "noalloc.cu", "tune.cu"]
CPP = ["setup_host.cpp"]


def _nvcc() -> str:
    for p in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if p and os.path.exists(p):
            return p
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(HERE, "..", "include")]
    jobs = []
    for f in CU:
        o = os.path.join(BUILD, f + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c",
               os.path.join(CSRC, f), "-o", o, *inc]
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        jobs.append((cmd, o))
    for f in CPP:
        o = os.path.join(BUILD, f + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-c", os.path.join(CSRC, f), "-o", o, *inc]
        jobs.append((cmd, o))
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(lambda j: _run(j[0]), jobs))
    link = [nvcc, *ARCH, "-shared", "-o", OUT + ".tmp", *[o for _, o in jobs], "-lcudart"]
    logs.append(_run(link))
    os.replace(OUT + ".tmp", OUT)
    if verbose:
        sys.stdout.write("".join(logs))
    return OUT


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv)
    print(OUT)
