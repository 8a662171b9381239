"""Build the native library ``libhlr_gb300.so`` in-tree (CUDA for sm_103a + C++ host code).

Each translation unit is compiled in parallel (nvcc for ``.cu``, g++ for ``.cpp``) into
``_build/`` and linked with nvcc into the package directory. Host code is compiled with
``-ffp-contract=off`` so that the encoder and the geometric predicates round like plain IEEE
code on every host architecture.
"""
from __future__ import annotations

import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhlr_gb300.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

CU = ["hlr_kernels.cu", "hlr_cg.cu", "hlr_encode.cu"]
CPP = ["hlr_codec.cpp", "hlr_upload.cpp", "hlr_pack.cpp", "hlr_build.cpp"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _cuda_home(nvcc: str) -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _sources_newer(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile (when sources changed) and return the path of the shared library."""
    nvcc = _nvcc()
    cuda = _cuda_home(nvcc)
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp.txt")
    want = f"{platform.machine()} {nvcc}\n"
    if not os.path.exists(stamp) or open(stamp).read() != want or not os.path.exists(LIB):
        force = True
    headers = [os.path.join(CSRC, "hlr_internal.h"), os.path.join(CSRC, "hlr_pack.h"), os.path.join(ROOT, "include", "hlr.h")]
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
    jobs = []
    objs = []
    for f in CU:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if force or _sources_newer(obj, [src] + headers):
            jobs.append([nvcc, ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                         "-Xptxas", "-v" if verbose else "-O3", *inc, "-c", src, "-o", obj])
    for f in CPP:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if force or _sources_newer(obj, [src] + headers):
            jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-ffp-contract=off",
                         "-I" + os.path.join(cuda, "include"), *inc, "-c", src, "-o", obj])
    procs = [(j, subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)) for j in jobs]
    failed = []
    for j, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out)
        if p.returncode != 0:
            failed.append((" ".join(j), out))
    if failed:
        msg = "\n".join(f"$ {c}\n{o}" for c, o in failed)
        raise RuntimeError("native build failed:\n" + msg)
    if force or jobs or _sources_newer(LIB, objs):
        link = [nvcc, ARCH, "-shared", "-o", LIB, *objs, "-Xcompiler", "-fopenmp", "-lgomp"]
        r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(link) + "\n" + r.stdout)
    with open(stamp, "w") as f:
        f.write(want)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
