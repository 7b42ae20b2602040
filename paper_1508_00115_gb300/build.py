"""Build libsph.so (the CUDA kernels + C-ABI) in-tree for sm_103a with nvcc.

Each translation unit compiles in parallel to an object, then nvcc links the
shared library next to this file.  No torch build machinery is involved; the
library links the CUDA runtime statically and depends on no Python.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsph.so")
SOURCES = ["sph_api.cu", "sph_cells.cu", "sph_pairs.cu", "sph_integrate.cu", "sph_tree.cu", "sph_hpredict.cu",
           "sph_gravity.cu", "sph_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "--extended-lambda",
         "-I", INCLUDE]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found (CUDA toolkit required to build libsph)")


# the pair kernels (k_density, k_force and their launches) and the cell and tree builds
# that lay out their work (cell order, leaves, the tiles' targets)
PAIR_SOURCES = ["sph_pairs.cu", "sph_internal.cuh", "sph_cells.cu", "sph_tree.cu"]


def _digest(files=None) -> str:
    """Identity of the sources (all of csrc/, or the given files of it), sph.h and
    the compile options."""
    h = hashlib.sha256()
    for f in sorted(files if files is not None else os.listdir(CSRC)):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    with open(os.path.join(INCLUDE, "sph.h"), "rb") as fh:
        h.update(fh.read())
    # the flags without the include directory's absolute path, so that the digest
    # names the sources and options, not the checkout's location
    h.update(" ".join(ARCH + [f for f in FLAGS if f != INCLUDE]).encode())
    return h.hexdigest()[:16]


GRAVITY_SOURCES = ["sph_gravity.cu", "sph_internal.cuh"]


def gravity_kernel_digest() -> str:
    """Identity of the gravity kernel's sources (ncu figures of k_gravity)."""
    return _digest(GRAVITY_SOURCES)


def pair_kernel_digest() -> str:
    """Identity of the pair kernels' sources and of the builds that lay out their work:
    ncu figures of k_density / k_force stay valid while it is unchanged."""
    return _digest(PAIR_SOURCES)


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a and link libsph.so; returns its path.
    Skips the work when the sources are unchanged since the last build."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == dig:
                return LIB
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_v else []

    def one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        res = list(ex.map(one, SOURCES))
    if verbose or ptxas_v:
        for _, err in res:
            if err:
                print(err)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in res], "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv))
