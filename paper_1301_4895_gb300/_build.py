"""In-tree build of libmbc.so (nvcc for sm_103a + g++ for the host builder).

Three translation units compiled in parallel, then linked with nvcc; no cmake.
The result lands next to this file and is git-ignored.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmbc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [
        os.path.join(HERE, "..", "include", "mbc.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(HERE, "..", "include")]
    cu_obj = os.path.join(OUT, "contract.o")
    cpp_obj = os.path.join(OUT, "builder.o")
    io_obj = os.path.join(OUT, "list_io.o")
    jobs = [
        [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", *inc, "-c",
         os.path.join(CSRC, "contract.cu"), "-o", cu_obj],
        ["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", *inc, "-c", os.path.join(CSRC, "builder.cpp"), "-o",
         cpp_obj],
        ["g++", "-O2", "-std=c++17", "-fPIC", *inc, "-c", os.path.join(CSRC, "list_io.cpp"), "-o", io_obj],
    ]

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)

    with ThreadPoolExecutor(max_workers=3) as ex:
        for f in [ex.submit(run, j) for j in jobs]:
            f.result()
    tmp = LIB + f".{os.getpid()}.tmp"
    run([nvcc, "-shared", *ARCH, "-o", tmp, cu_obj, cpp_obj, io_obj, "-Xcompiler", "-fopenmp", "-lgomp"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
