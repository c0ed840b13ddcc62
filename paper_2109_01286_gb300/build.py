"""Builds the in-tree shared library `_lib/libhfd.so` (CUDA for sm_103a + host C++).

Three translation units compile in parallel: csrc/prep.cpp (g++), csrc/kernels.cu and
csrc/api.cu (nvcc, -gencode arch=compute_103a,code=sm_103a), then nvcc links them with the
CUDA runtime.  Host code is built with -ffp-contract=off (see csrc/prep.cpp) and without
machine-specific flags, so the x86 and Arm builds compute the same host results.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libhfd.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _sources():
    return [os.path.join(CSRC, f) for f in ("prep.cpp", "kernels.cu", "api.cu", "noalloc.cu",
                                            "adjoint.cu")]


def _deps():
    return _sources() + [os.path.join(CSRC, f) for f in ("prep.hpp", "kernels.hpp", "mesh.hpp",
                                                         "adjoint_kernels.cuh")] + \
        [os.path.join(INCLUDE, "hfd.h"), os.path.abspath(__file__)]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force=False, verbose=False):
    """Compile and link libhfd.so unless it is newer than every source."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    bdir = os.path.join(OUT_DIR, "obj")
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    common = ["-std=c++17", "-O3", f"-I{INCLUDE}", f"-I{CSRC}"]
    cmds = []
    objs = []
    for src in _sources():
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        objs.append(obj)
        if src.endswith(".cpp"):
            cmds.append(["g++", "-fPIC", "-ffp-contract=off", "-pthread", "-Wall"] + common +
                        ["-c", src, "-o", obj])
        else:
            cmds.append([nvcc, ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off"] +
                        common + ["-c", src, "-o", obj])
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
             for c in cmds]
    failed = []
    for c, p in zip(cmds, procs):
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out)
        if p.returncode != 0:
            failed.append((" ".join(c), out))
    if failed:
        msg = "\n".join(f"$ {c}\n{o}" for c, o in failed)
        raise RuntimeError(f"libhfd build failed:\n{msg}")
    tmp = LIB + ".tmp"
    link = [nvcc, ARCH, "-shared", "-o", tmp] + objs + ["-lcudart", "-lpthread"]
    p = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"libhfd link failed:\n$ {' '.join(link)}\n{p.stdout}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
