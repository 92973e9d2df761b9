"""Builds libhd.so (the C-ABI library with the sm_103a decode kernels) in-tree.

Every translation unit is compiled by nvcc for ``sm_103a`` only, in parallel,
then linked into ``paper_2201_09118_gb300/_build/libhd.so``.  The CUDA runtime
is linked statically so the library does not depend on which libcudart the
host process (e.g. PyTorch) loaded.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhd.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def nvcc() -> str:
    path = shutil.which("nvcc")
    if path:
        return path
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhd.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(
        os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [__file__]


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), out_dir: str = None) -> str:
    """Compile and link libhd.so if any source changed; returns its path.

    ``extra_flags``/``out_dir`` build a variant elsewhere (extra nvcc flags,
    another directory); the default build goes to _build/libhd.so."""
    build_dir = out_dir or BUILD
    lib = os.path.join(build_dir, "libhd.so")
    with _lock:
        if not force and not _stale(lib):
            return lib
        os.makedirs(os.path.join(build_dir, "obj"), exist_ok=True)
        cc = nvcc()
        common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                         "-I", INCLUDE, "-I", CSRC, *extra_flags]

        def compile_one(src):
            obj = os.path.join(build_dir, "obj", os.path.basename(src) + ".o")
            cmd = [cc, *common, "-c", src, "-o", obj]
            if src.endswith(".cpp"):
                cmd = [cc, "-x", "cu", *common, "-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
            if verbose and r.stderr:
                print(r.stderr)
            return obj

        srcs = _sources()
        with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
            objs = list(ex.map(compile_one, srcs))
        tmp = lib + f".tmp{os.getpid()}"
        r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
        return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
