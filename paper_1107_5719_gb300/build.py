"""Build librt3d.so in-tree with nvcc for sm_103a (GB300).

The translation units under ``csrc/`` are compiled in parallel into
``_build/`` and linked into ``librt3d.so`` next to this file.  No cmake, no
torch extension machinery: the library has a plain C ABI.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librt3d.so")
# The checked build (-DRT_CHECKED): bounds tests on every gathered index of
# the marches and stencils, reported as RT_EBOUNDS; loaded instead of LIB
# when RT3D_CHECKED=1.
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "librt3d_checked.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["fs.cu", "fs32.cu", "fsdf.cu", "sc.cu", "para.cu", "os.cu", "api.cu", "noalloc.cu",
           "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librt3d.so")
    return path


def _deps():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, "internal.h"), os.path.join(CSRC, "weights.cuh"),
              os.path.join(CSRC, "df.cuh"),
              os.path.join(INCLUDE, "rt3d.h")]
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    """Compile and link librt3d.so (or librt3d_checked.so); returns its path."""
    return build_many([checked], force, verbose, extra_flags)[0]


def build_many(variants=(False, True), force: bool = False, verbose: bool = False,
               extra_flags=()) -> list:
    """Compile the requested variants (False: normal, True: checked) with all
    translation units of all variants in one parallel pool."""
    cc = nvcc()
    todo = [v for v in variants if force or not up_to_date(LIB_CHECKED if v else LIB)]
    jobs = []
    for v in todo:
        os.makedirs(BUILD_CHECKED if v else BUILD, exist_ok=True)
        jobs += [(v, src) for src in SOURCES]

    def compile_one(job):
        v, src = job
        obj = os.path.join(BUILD_CHECKED if v else BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra_flags, *(["-DRT_CHECKED"] if v else []),
               "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        objs = list(ex.map(compile_one, jobs))
    for v in todo:
        lib = LIB_CHECKED if v else LIB
        mine = [o for (vv, _), o in zip(jobs, objs) if vv == v]
        tmp = lib + f".{os.getpid()}.tmp"
        r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *mine], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return [LIB_CHECKED if v else LIB for v in variants]


if __name__ == "__main__":
    print(build_many(force="--force" in sys.argv, verbose="-v" in sys.argv))
