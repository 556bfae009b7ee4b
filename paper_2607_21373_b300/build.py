"""Builds libpat.so in-tree with nvcc for sm_103a (no JIT cache, no torch types).

Every source is compiled to an object in parallel (whole-program device code per
file, as one nvcc command would), then the objects are linked into the shared
library."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpat.so")
SOURCES = ["pat_host.cpp", "pat_kernels.cu", "pat_grad.cu", "pat_multi.cu", "pat_noalloc.cu", "pat_matern.cu",
           "pat_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = [*ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp,-O3", "-Xptxas", "-v"]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "pat.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libpat.so if a source is newer than the library; returns its path."""
    if not force and not needs_build():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    with tempfile.TemporaryDirectory() as tmp:
        objs = [os.path.join(tmp, os.path.splitext(s)[0] + ".o") for s in SOURCES]

        def compile_one(i):
            cmd = [nvcc, *NVCC_FLAGS, "-c", os.path.join(CSRC, SOURCES[i]), "-o", objs[i]]
            return subprocess.run(cmd, capture_output=True, text=True)

        with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            results = list(ex.map(compile_one, range(len(SOURCES))))
        log = "".join(r.stdout + r.stderr for r in results)
        if any(r.returncode != 0 for r in results):
            sys.stderr.write(log)
            raise RuntimeError("nvcc failed building libpat.so")
        link = subprocess.run([nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *objs, "-lgomp"], capture_output=True,
                              text=True)
        if link.returncode != 0:
            sys.stderr.write(link.stdout + link.stderr)
            raise RuntimeError("nvcc failed linking libpat.so")
    if verbose:
        sys.stderr.write(log)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
