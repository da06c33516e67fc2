"""Build libitm.so in-tree for sm_103a with nvcc.

Each translation unit is compiled separately (in parallel) and linked into
``paper_1708_00783_gb300/_lib/libitm.so``.  The kernels that decide integers
from floats (allocation, integration, raycast) rely on IEEE round-to-nearest
intrinsics; ``-fmad=false`` and the host's ``-ffp-contract=off`` keep any
other float expression unfused as well.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ_DIR = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIB_DIR, "libitm.so")
# the bounds-checked debug build (-DITM_CHECK_BOUNDS): index checks before
# the accesses of the hot kernels, a failed check reported as ITM_ERR_BOUNDS
OBJ_DIR_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(LIB_DIR, "libitm_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", INCLUDE,
          "-I", CSRC, "--expt-relaxed-constexpr"]
# per translation unit extra flags
SOURCES = {
    "itm_scene.cu": ["-fmad=false"],
    "itm_alloc.cu": ["-fmad=false"],
    "itm_integrate.cu": ["-fmad=false"],
    "itm_raycast.cu": ["-fmad=false"],
    "itm_depth.cu": ["-fmad=false"],
    "itm_noalloc.cu": ["-fmad=false"],
    "itm_conf.cu": [],
    "itm_batch.cu": ["-fmad=false"],
    "itm_combined.cu": ["-fmad=false"],
    "itm_swap.cu": ["-fmad=false"],
    "itm_colour.cu": ["-fmad=false"],
    "itm_track.cu": ["-fmad=false"],
    "itm_mesh.cu": ["-fmad=false"],
}


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _deps_mtime() -> float:
    m = os.path.getmtime(os.path.join(INCLUDE, "itm.h"))
    for f in os.listdir(CSRC):
        m = max(m, os.path.getmtime(os.path.join(CSRC, f)))
    return max(m, os.path.getmtime(__file__))


def build(force: bool = False, verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    obj_dir, lib_path = (OBJ_DIR_CHECKED, LIB_CHECKED) if checked else (OBJ_DIR, LIB)
    if checked:
        extra_flags = tuple(extra_flags) + ("-DITM_CHECK_BOUNDS",)
    os.makedirs(obj_dir, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= _deps_mtime():
        return lib_path
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *SOURCES[src], *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr))
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, sorted(SOURCES)))
    tmp = lib_path + ".%d.tmp" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr)
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
