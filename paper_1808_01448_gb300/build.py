"""In-tree build of the CUDA library ``_build/liblbib.so`` for sm_103a, and of
its bounds-checked debug form ``_build/liblbib_debug.so`` (``-DLBIB_DEBUG``:
every population index of the lattice and particle passes is checked, a
failed check is reported as LBIB_E_BOUNDS).

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library with the CUDA runtime linked statically.  Nothing is
installed outside this directory.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbib.so")
LIB_DEBUG = os.path.join(BUILD, "liblbib_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbib.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(ROOT, "include", "lbib.h"), __file__]


def up_to_date(path: str = LIB) -> bool:
    if not os.path.exists(path):
        return False
    t = os.path.getmtime(path)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool | None = None) -> str:
    """Compile and link the libraries whose sources are newer; returns the
    release library's path.  debug: None builds both forms, True or False
    only the debug or the release one."""
    forms = [(LIB, False), (LIB_DEBUG, True)]
    if debug is not None:
        forms = [f for f in forms if f[1] == debug]
    todo = [(path, dbg) for path, dbg in forms if force or not up_to_date(path)]
    if not todo:
        return LIB
    os.makedirs(os.path.join(BUILD, "debug"), exist_ok=True)
    cc = nvcc()

    def compile_one(job):
        src, dbg = job
        odir = os.path.join(BUILD, "debug") if dbg else BUILD
        obj = os.path.join(odir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *FLAGS, *ARCH, *(["-DLBIB_DEBUG"] if dbg else []), "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return dbg, obj

    jobs = [(src, dbg) for _, dbg in todo for src in sources()]
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        done = list(ex.map(compile_one, jobs))
    for path, dbg in todo:
        objs = [o for d, o in done if d == dbg]
        tmp = path + f".tmp{os.getpid()}"
        r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, path)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
