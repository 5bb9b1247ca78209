"""Build libsdfgjacobi.so in-tree (``paper_1902_10345_gb300/_build/``).

CUDA sources compile for sm_103a only (``-gencode arch=compute_103a,code=sm_103a``);
host sources compile with g++.  Translation units build in parallel and the
library is relinked only when a source or header changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsdfgjacobi.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                     "-Xptxas", "-warn-spills"]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function"]
# developer knobs: SDFG_DEFINES (e.g. "-DSDFG_CHUNK_ROWS=12 -DSDFG_STAGES=2") reaches BOTH
# compilers, so host planning and kernels agree on shared constants;
# SDFG_NVCC_EXTRA adds device-only flags (e.g. -DSDFG_TP_MINB=4)
_DEFINES = os.environ.get("SDFG_DEFINES", "").split()
NVCC_FLAGS += _DEFINES + os.environ.get("SDFG_NVCC_EXTRA", "").split()
CXX_FLAGS += _DEFINES


def cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _digest() -> str:
    h = hashlib.sha256()
    files = _sources() + sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")))
    files += sorted(glob.glob(os.path.join(INCLUDE, "*.h")))
    for f in files:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS + CXX_FLAGS).encode())
    return h.hexdigest()


KERNEL_FILES = ["device_common.cuh", "temporal_unit.cuh", "geometry.h", "persistent.h", "persistent.cu", "kernels.cu"]
KERNEL_FILES_3D = ["device_common.cuh", "jacobi3d.cu"]
KERNEL_FILES_SOR = ["device_common.cuh", "sor2d.cu"]
KERNEL_FILES_RESIDENT = ["device_common.cuh", "resident.cu"]
KERNEL_FILES_CHAIN = ["device_common.cuh", "temporal_unit.cuh", "geometry.h", "chain.cuh", "skewed.cu", "chain_batch.cu"]


_TOKENS = re.compile(r'"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'|//[^\n]*|/\*.*?\*/', re.S)


def _code_only(text: str) -> str:
    """C/C++/CUDA source without comments and with whitespace runs collapsed
    (string and character literals, such as inline PTX, are kept)."""
    text = _TOKENS.sub(lambda m: " " if m.group(0).startswith("/") else m.group(0), text)
    return " ".join(text.split())


def kernel_digest(files=None) -> str:
    """Digest of the device sources and flags that define the kernels (used
    to tell whether a committed profile still describes the current kernels);
    comments and layout do not count.  files: the 2-D kernels' sources by
    default, KERNEL_FILES_3D, KERNEL_FILES_SOR, KERNEL_FILES_RESIDENT or
    KERNEL_FILES_CHAIN for the 3-D, SOR, register-resident and chain kernels."""
    h = hashlib.sha256()
    for f in files or KERNEL_FILES:
        with open(os.path.join(CSRC, f), encoding="utf-8") as fh:
            h.update(f.encode())
            h.update(_code_only(fh.read()).encode())
    h.update(" ".join(NVCC_FLAGS).encode())
    return h.hexdigest()[:16]


def _compile(src: str, cuda: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, "obj", os.path.basename(src) + ".o")
    inc = ["-I" + CSRC, "-I" + INCLUDE, "-I" + os.path.join(cuda, "include")]
    if src.endswith(".cu"):
        cmd = [os.path.join(cuda, "bin", "nvcc"), *NVCC_FLAGS, *inc, "-c", src, "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
    else:
        cmd = ["g++", *CXX_FLAGS, *inc, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stderr or r.stdout):
        sys.stderr.write(r.stdout + r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link the library if anything changed; return its path."""
    os.makedirs(os.path.join(BUILD, "obj"), exist_ok=True)
    stamp = os.path.join(BUILD, "stamp.txt")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    cuda = cuda_home()
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, cuda, verbose), srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [os.path.join(cuda, "bin", "nvcc"), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
