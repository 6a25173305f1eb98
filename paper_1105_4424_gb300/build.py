"""Builds the in-tree CUDA library ``libarol.so`` for sm_103a with nvcc.

Translation units are compiled in parallel (one nvcc per file, one
``-gencode``) and linked into a shared library with the CUDA runtime linked
statically, so the library loads without any other CUDA shared object.
"""
from __future__ import annotations

import glob
import os
import platform
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libarol.so")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE, "-I", CSRC,
         "--expt-relaxed-constexpr"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, extra):
    obj = os.path.join(OBJDIR, os.path.basename(src) + ".o")
    if _stale(obj, [src] + _headers()):
        cmd = [NVCC] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, extra_flags=None, verbose: bool = False) -> str:
    """Compile every translation unit under csrc/ and link libarol.so."""
    os.makedirs(OBJDIR, exist_ok=True)
    stamp = os.path.join(OBJDIR, "arch.txt")
    arch = platform.machine()
    if not os.path.exists(stamp) or open(stamp).read().strip() != arch:
        force = True   # objects of another host architecture
    extra = list(extra_flags or [])
    srcs = _sources()
    if force:
        for o in glob.glob(os.path.join(OBJDIR, "*.o")):
            os.remove(o)
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs))
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(arch + "\n")
    if verbose:
        print(f"built {LIB}")
    return LIB


DEBUG_LIB = os.path.join(PKG, "libarol_debug.so")
DEBUG_SOURCES = ("k_tiler.cu",)   # the units whose AROL_DEBUG checks differ


def build_debug(verbose: bool = False) -> str:
    """libarol_debug.so: the release objects, except that the units in
    DEBUG_SOURCES are compiled with -DAROL_DEBUG (device-side bounds checks
    on every index of the per-repetition walk, reported as AROL_ERR_OOB).
    Load it with AROL_LIB=<path> before importing the package."""
    build()
    dbgdir = os.path.join(OBJDIR, "debug")
    os.makedirs(dbgdir, exist_ok=True)
    objs = []
    for src in _sources():
        name = os.path.basename(src)
        if name in DEBUG_SOURCES:
            obj = os.path.join(dbgdir, name + ".o")
            if _stale(obj, [src] + _headers()):
                cmd = [NVCC] + ARCH + FLAGS + ["-DAROL_DEBUG", "-c", src, "-o", obj]
                r = subprocess.run(cmd, capture_output=True, text=True)
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed on {name}:\n{r.stdout}\n{r.stderr}")
            objs.append(obj)
        else:
            objs.append(os.path.join(OBJDIR, name + ".o"))
    if _stale(DEBUG_LIB, objs):
        tmp = DEBUG_LIB + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, DEBUG_LIB)
    if verbose:
        print(f"built {DEBUG_LIB}")
    return DEBUG_LIB


if __name__ == "__main__":
    build(verbose=True)
