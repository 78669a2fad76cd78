"""Build the device libraries in-tree (sm_103a only): the query library
csrc/*.cu -> _build/librt_gb300.so, and the measurement probes
csrc/probe/mem_probe.cu -> _build/libmem_probe.so.

Translation units compile in parallel; only changed ones are rebuilt.  Run as
`python -m paper_2305_07253_gb300.build` or through `__graft_entry__.build()`.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "librt_gb300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["rt_api.cu", "rt_scene.cu", "rt_treelet.cu", "rt_wide.cu", "rt_bake.cu", "rt_dfgen.cu", "rt_trace.cu",
           "rt_backward.cu", "rt_batch.cu", "rt_order.cu"]
PROBE_SOURCE = os.path.join("probe", "mem_probe.cu")
PROBE_LIB = os.path.join(OUT, "libmem_probe.so")
HEADERS = ["rt_internal.cuh", "rt_trace_dev.cuh", "rt_bake_dev.cuh"]

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC,-O2,-ffp-contract=off",
    "-I", INCLUDE,
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "rt_api.h"),
                                                        os.path.join(INCLUDE, "mem_probe.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(OUT, os.path.basename(src).replace(".cu", ".o"))
    s = os.path.join(CSRC, src)
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(s), _deps_mtime()):
        return obj
    cmd = [nvcc(), *NVCC_FLAGS, "-c", s, "-o", obj + ".tmp"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def _link(lib: str, objs: list, verbose: bool) -> str:
    if os.path.exists(lib) and os.path.getmtime(lib) >= max(os.path.getmtime(o) for o in objs):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build(verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES + [PROBE_SOURCE]))
    _link(PROBE_LIB, objs[-1:], verbose)
    return _link(LIB, objs[:-1], verbose)


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
