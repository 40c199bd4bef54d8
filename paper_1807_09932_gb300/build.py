"""Build the EBIC GB300 CUDA library in-tree (nvcc, sm_103a only).

Every translation unit under ``csrc/`` is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` (no fast-math: the rank transform
orders IEEE bit patterns and must not flush subnormals) and linked, with the CUDA runtime
linked statically, into ``lib/libebic_gb300.so``. The library needs no libcuda at link time:
the one driver entry point it uses (tensor-map encoding) is fetched at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys
import sysconfig

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(PKG, "_build")
LIB_DIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIB_DIR, "libebic_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", INCLUDE, "-I", CSRC]


PYFAST_SRC = os.path.join(CSRC, "pyfast.c")


def pyfast_path() -> str:
    """Where the C marshalling module for the per-generation calls is built."""
    return os.path.join(LIB_DIR, "_ebic_fast" + (sysconfig.get_config_var("EXT_SUFFIX") or ".so"))


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, verbose_ptxas=False):
    obj = os.path.join(OBJ, os.path.basename(src) + ".o")
    if not _stale(obj, [src, __file__] + _headers()):
        return obj, ""
    cmd = [nvcc(), "-c", src, "-o", obj] + ARCH + FLAGS
    if verbose_ptxas and src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None) -> str:
    """Compile and link the library if any source changed. Returns the library path."""
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    if force:
        for f in glob.glob(os.path.join(OBJ, "*.o")):
            os.remove(f)
    srcs = _sources()
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    logs = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose_ptxas), srcs))
    objs = [o for o, _ in results]
    logs = [l for _, l in results if l]
    if _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    _build_pyfast()
    if verbose_ptxas:
        sys.stderr.write("\n".join(logs))
    return LIB


def _build_pyfast():
    """The CPython module that converts the per-generation calls' arguments in C (linked to the
    library beside it). Built only where the interpreter's headers are installed; without it the
    binding converts the same arguments through ctypes."""
    inc = sysconfig.get_paths().get("include") or ""
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc or not os.path.exists(os.path.join(inc, "Python.h")):
        return None
    out = pyfast_path()
    if not _stale(out, [PYFAST_SRC, os.path.join(INCLUDE, "ebic.h"), __file__, LIB]):
        return out
    tmp = out + f".{os.getpid()}.tmp"
    cmd = [cc, "-shared", "-fPIC", "-O2", "-std=c11", "-Wall", "-I", inc, "-I", INCLUDE,
           PYFAST_SRC, "-L", LIB_DIR, "-lebic_gb300", "-Wl,-rpath,$ORIGIN", "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"building the marshalling module failed:\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
