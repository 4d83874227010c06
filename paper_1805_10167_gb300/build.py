"""Build libhhg.so in place: every translation unit under csrc/ compiled by
nvcc for sm_103a (in parallel), then linked into one shared library next to
this file.  With checked=True (--checked) it builds libhhg_checked.so
instead: the translation units whose kernels carry device-side index checks
are recompiled with -DHHG_CHECK_BOUNDS, the other objects of the normal
build are reused.  Usage: python -m paper_1805_10167_gb300.build [--jobs N]
[--checked]."""
from __future__ import annotations

import os
import re
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libhhg.so")
OUT_CHECKED = os.path.join(HERE, "libhhg_checked.so")
BUILD = os.path.join(HERE, "_build")
BUILD_CHECKED = os.path.join(BUILD, "checked")
# the checked index helpers of hhg_internal.h (and the row functions that use them)
_CHECKED_USE = re.compile(r"\b(face_id|edge_id|vert_id|edge_pos|table_range|face_task|frame_slot|frame_up|frame_dn)\(|"
                          r'#include "stencil\.cuh"')
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def uses_checks(src):
    with open(src) as f:
        return src.endswith(".cu") and _CHECKED_USE.search(f.read()) is not None


def _compile(src, checked=False):
    obj = os.path.join(BUILD_CHECKED if checked else BUILD, os.path.basename(src) + ".o")
    lang = ["-x", "cu"] if src.endswith(".cu") else ["-x", "c++"]
    extra = ["-DHHG_CHECK_BOUNDS"] if checked else []
    cmd = [NVCC] + ARCH + FLAGS + extra + lang + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    return obj


def build(jobs: int | None = None, verbose: bool = False, checked: bool = False) -> str:
    os.makedirs(BUILD_CHECKED if checked else BUILD, exist_ok=True)
    srcs = sources()
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    if checked:
        redo = [s for s in srcs if uses_checks(s)]
        reuse = {s: os.path.join(BUILD, os.path.basename(s) + ".o") for s in srcs if s not in redo}
        missing = [s for s, o in reuse.items() if not os.path.exists(o)]
        with ThreadPoolExecutor(max_workers=jobs) as ex:
            done = dict(zip(redo, ex.map(lambda s: _compile(s, True), redo)))
            done.update(zip(missing, ex.map(_compile, missing)))
        objs = [done.get(s, reuse.get(s)) for s in srcs]
        out = OUT_CHECKED
    else:
        with ThreadPoolExecutor(max_workers=jobs) as ex:
            objs = list(ex.map(_compile, srcs))
        out = OUT
    cmd = [NVCC] + ARCH + ["-shared", "-o", out] + objs + ["-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    if verbose:
        print("built", out)
    return out


if __name__ == "__main__":
    jobs = int(sys.argv[sys.argv.index("--jobs") + 1]) if "--jobs" in sys.argv else None
    build(jobs, verbose=True, checked="--checked" in sys.argv)
