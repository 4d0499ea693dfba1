"""Build libnanobte.so in-tree with nvcc for sm_103a (no GPU needed), and
libnanobte_checks.so, the same library with the sweep's device-side
consistency checks compiled in (NBTE_CHECKS: index bounds, level order and
ring-slot reuse, reported as an error status instead of a fault).

    python -m paper_2607_03226_b300.build [--force] [--checks]
"""
from __future__ import annotations

import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libnanobte.so")
LIB_CHECKS = os.path.join(HERE, "libnanobte_checks.so")
BUILD = os.path.join(HERE, "_build")

SOURCES = ["mesh.cpp", "plan.cpp", "coarse.cpp", "capi.cpp", "kernels.cu", "sweep.cu", "sweep_data.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _digest():
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)) + ["../../include/nbte.h"]:
        p = os.path.join(CSRC, name)
        if os.path.isfile(p):
            with open(p, "rb") as f:
                h.update(name.encode() + f.read())
    h.update(" ".join(ARCH).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    lib = LIB_CHECKS if checks else LIB
    bdir = os.path.join(BUILD, "checks") if checks else BUILD
    os.makedirs(bdir, exist_ok=True)
    stamp = os.path.join(bdir, "stamp")
    dg = _digest()
    if not force and os.path.exists(lib) and os.path.exists(stamp) and open(stamp).read() == dg:
        return lib
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-Xcompiler", "-fPIC", "-lineinfo"]
    if checks:
        common.append("-DNBTE_CHECKS")

    def compile_one(src):
        obj = os.path.join(bdir, src + ".o")
        cmd = [NVCC, *common, *ARCH, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu") and verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, obj, cmd, r

    # the translation units are independent: compile them side by side
    workers = max(1, min(len(SOURCES), os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(compile_one, SOURCES))
    objs = []
    for src, obj, cmd, r in results:
        if verbose:
            print(" ".join(cmd))
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        objs.append(obj)
    cmd = [NVCC, "-shared", *ARCH, "-o", lib, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    with open(stamp, "w") as f:
        f.write(dg)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checks="--checks" in sys.argv))
