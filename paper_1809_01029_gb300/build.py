"""Build libpyjac_gb.so in-tree for sm_103a (nvcc; translation units compiled
in parallel).  Usage: ``python -m paper_1809_01029_gb300.build``."""
from __future__ import annotations

import os
import subprocess
import sys
import time
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libpyjac_gb.so")
# the bounds-checked build (index-table lookups checked into a device error
# word, see include/pyjac_gb.h: pj_debug_word)
BUILD_DBG = os.path.join(PKG, "_build_dbg")
LIB_DBG = os.path.join(LIBDIR, "libpyjac_gb_dbg.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["mech.cpp", "api.cpp", "kinetics.cu", "noalloc.cu", "forms.cu", "batch.cu", "fd.cu", "lu.cu", "lu_symbolic.cpp", "hostio.cpp"]
# jacobian_inst.cu is compiled once per (layout, precision): object name,
# then its defines (see the file's header)
JAC_INSTANCES = [
    (f"jac_{lay}_{prec}", {"PJ_INST_TM": tm, "PJ_INST_F32": int(prec == "f32"),
                           "PJ_INST_NAME": f"launch_jac_{lay}_{prec}"})
    for lay, tm in (("plain", -1), ("tm0", 0), ("tm1", 1), ("tm2", 2), ("coop", 3))
    for prec in ("f64", "f32")
]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "pyjac_gb.h"))
    return files


def up_to_date(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def _compile(job) -> str:
    src, name, defs, build_dir = job
    obj = os.path.join(build_dir, name + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
           *[f"-D{k}={v}" for k, v in defs.items()],
           "-I", INCLUDE, "-I", CSRC, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, debug_bounds: bool = False) -> str:
    """Compile every translation unit and link the shared library
    (debug_bounds: the bounds-checked variant, LIB_DBG)."""
    lib, build_dir = (LIB_DBG, BUILD_DBG) if debug_bounds else (LIB, BUILD)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    extra = {"PJ_DEBUG_BOUNDS": 1} if debug_bounds else {}
    jobs = [(s, s, dict(extra), build_dir) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    jobs += [("jacobian_inst.cu", name, {**defs, **extra}, build_dir) for name, defs in JAC_INSTANCES]
    t0 = time.time()
    with ThreadPoolExecutor(max_workers=min(len(jobs), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(_compile, jobs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib} in {time.time() - t0:.1f}s", file=sys.stderr)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, debug_bounds="--debug-bounds" in sys.argv)
