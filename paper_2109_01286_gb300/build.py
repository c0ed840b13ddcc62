"""Builds the in-tree shared libraries `_lib/libhfd.so` (CUDA for sm_103a + host C++) and
`_lib/libhfd_check.so`, the bounds-checked build of the same library.

The translation units compile in parallel: csrc/prep.cpp and csrc/prep3.cpp (g++), the .cu files (nvcc,
-gencode arch=compute_103a,code=sm_103a), and csrc/kernels.cu once more with -DHFD_CHECK=1
(every gathered index tested on the device, see chk_idx in kernels.cu); then nvcc links each
library with the CUDA runtime.  Host code is built with -ffp-contract=off (see csrc/prep.cpp) and without
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
LIB_CHECK = os.path.join(OUT_DIR, "libhfd_check.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _sources():
    return [os.path.join(CSRC, f) for f in ("prep.cpp", "kernels.cu", "api.cu", "noalloc.cu",
                                            "adjoint.cu", "peaks.cu", "prep3.cpp", "kernels3d.cu",
                                            "api3d.cu")]


def _deps():
    return _sources() + [os.path.join(CSRC, f) for f in ("prep.hpp", "kernels.hpp", "mesh.hpp",
                                                         "adjoint_kernels.cuh", "linalg.hpp",
                                                         "mesh3.hpp", "kernels3d.hpp", "fp_convert.cuh")] + \
        [os.path.join(INCLUDE, "hfd.h"), os.path.join(INCLUDE, "hfd3d.h"), os.path.abspath(__file__)]


def up_to_date():
    if not (os.path.exists(LIB) and os.path.exists(LIB_CHECK)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_CHECK))
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
    kcheck = os.path.join(bdir, "kernels_check.cu.o")
    cmds.append([nvcc, ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off", "-DHFD_CHECK=1"] +
                common + ["-c", os.path.join(CSRC, "kernels.cu"), "-o", kcheck])
    objs_check = [kcheck if o.endswith(os.sep + "kernels.cu.o") else o for o in objs]
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
    for out, ob in ((LIB_CHECK, objs_check), (LIB, objs)):
        tmp = out + ".tmp"
        link = [nvcc, ARCH, "-shared", "-o", tmp] + ob + ["-lcudart", "-lpthread"]
        p = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"{os.path.basename(out)} link failed:\n$ {' '.join(link)}\n{p.stdout}")
        os.replace(tmp, out)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
