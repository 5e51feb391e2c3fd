"""Build the CUDA library ``libvlb.so`` in-tree for sm_103a with nvcc.

Each translation unit under ``csrc/`` compiles in parallel to an object file
under ``_build/``; the objects link into ``paper_2410_23802_gb300/libvlb.so``.
The CUDA runtime is linked statically, so loading the library needs only the
driver (and no GPU until the first CUDA call).
"""
from __future__ import annotations

import concurrent.futures
import json
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libvlb.so")
SOURCES = ["vlb_lattice.cu", "vlb_particles.cu", "vlb_batch.cu", "vlb_capi.cu", "vlb_noalloc.cu", "vlb_serve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvlb.so")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


TUNED = os.path.join(PKG, "tuned.json")


def tuned_defines(path: str = TUNED) -> list[str]:
    """The build-time shape the autotuner chose (``autotune.py``): the
    ``defines`` of the entry named by ``use`` in tuned.json, else none."""
    try:
        with open(path) as fh:
            rec = json.load(fh)
        return list(rec[rec["use"]]["defines"])
    except (OSError, KeyError, ValueError, TypeError):
        return []


def build(verbose: bool = False, force: bool = False, defines: list[str] | None = None,
          out: str | None = None) -> str:
    """Compile (if needed) and return the path of the library.

    Preprocessor definitions (tile height VLB_TILE_Y, VLB_LATTICE_MIN_BLOCKS)
    come from `defines`, else from the environment variable VLB_DEFINES, else
    from the autotuner's tuned.json; a change of them forces a rebuild.
    `out` builds a library of another name (objects in a folder of its own)."""
    nvcc = _nvcc()
    lib = out or LIB
    bdir = BUILD if out is None else os.path.join(BUILD, os.path.splitext(os.path.basename(out))[0])
    os.makedirs(bdir, exist_ok=True)
    if defines is None:
        env = os.environ.get("VLB_DEFINES")
        defines = env.split() if env is not None else tuned_defines()
    defines = ["-D" + d for d in defines]
    stamp = os.path.join(bdir, "defines.txt")
    old = open(stamp).read() if os.path.exists(stamp) else ""
    if old != " ".join(defines):
        force = True
        with open(stamp, "w") as fh:
            fh.write(" ".join(defines))
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "vlb.h"))
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc, *ARCH, *FLAGS, *defines, "-I", os.path.join(ROOT, "include"), "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {cmd[-3]}")

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _stale(lib, objs):
        tmp = lib + ".tmp"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
