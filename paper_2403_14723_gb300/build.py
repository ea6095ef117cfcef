"""Build libpolylla (the sm_103a CUDA library) in-tree with nvcc.

The translation units under ``csrc/`` compile in parallel to objects and
link into ``_build/<machine>/libpolylla.so``.  A content hash of the sources
and flags names the build, so an unchanged tree is not rebuilt.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
SOURCES = ["polylla_api.cu", "kernels_label.cu", "kernels_repair.cu", "kernels_output.cu", "kernels_batch.cu",
           "kernels_serve.cu", "polylla_noalloc.cu", "polylla_server.cu", "kernels_lepp.cu", "kernels_convex.cu"]
HEADERS = [os.path.join(CSRC, "polylla_internal.cuh"), os.path.join(CSRC, "polylla_serve.cuh"),
           os.path.join(CSRC, "serve_policy.h"), os.path.join(INCLUDE, "polylla.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I" + INCLUDE]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpolylla")


# the files that define the method's kernels (their DRAM traffic, recorded
# from ncu, stays valid while these are unchanged)
CORE_SOURCES = ["kernels_label.cu", "kernels_repair.cu", "kernels_output.cu", "polylla_internal.cuh"]


def core_digest() -> str:
    """Digest of the method's kernel sources and compile flags."""
    h = hashlib.sha1()
    for s in CORE_SOURCES:
        with open(os.path.join(CSRC, s), "rb") as fh:
            h.update(fh.read())
    flags = [f for f in NVCC_FLAGS if not f.startswith("-I")]
    h.update(" ".join(ARCH + flags).encode())
    return h.hexdigest()[:12]


def _digest(extra=()) -> str:
    h = hashlib.sha1()
    for f in [os.path.join(CSRC, s) for s in SOURCES] + HEADERS:
        with open(f, "rb") as fh:
            h.update(fh.read())
    # the include directory is an absolute path that differs between
    # checkouts; leave it out so a source digest is the same everywhere
    flags = [f for f in NVCC_FLAGS if not f.startswith("-I")]
    h.update(" ".join(ARCH + flags + list(extra)).encode())
    return h.hexdigest()[:12]


def build_dir() -> str:
    return os.path.join(PKG, "_build", platform.machine())


def library_path() -> str:
    return os.path.join(build_dir(), "libpolylla.so")


def build_library(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every CUDA source for sm_103a and link libpolylla.so."""
    out = library_path()
    stamp = out + ".stamp"
    dig = _digest(["-Xptxas=-v"] if ptxas_info else [])
    if not force and os.path.exists(out) and os.path.exists(stamp) and open(stamp).read() == dig:
        return out
    os.makedirs(build_dir(), exist_ok=True)
    nvcc = nvcc_path()
    flags = ARCH + NVCC_FLAGS + (["-Xptxas", "-v"] if ptxas_info else [])

    def compile_one(src):
        obj = os.path.join(build_dir(), src.replace(".cu", ".o"))
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for _, err in results:
            if err:
                print(err)
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc, "-shared", "-o", tmp] + [o for o, _ in results] + ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, out)
    with open(stamp, "w") as f:
        f.write(dig)
    return out


if __name__ == "__main__":
    import sys

    print(build_library(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
