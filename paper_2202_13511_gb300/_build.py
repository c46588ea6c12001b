"""Build of the CUDA library ``libmpdp.so`` for sm_103a (in-tree, no cmake).

Each translation unit is compiled by its own nvcc process in parallel, then
linked into one shared library with a plain C ABI (``include/mpdp.h``).
Device code is built with ``-fmad=false`` so that no multiply-add is ever
contracted: the DP's floating-point results must match IEEE operations done
one at a time.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libmpdp.so")
# the multi-threaded CPU MPDP (a comparison baseline; plain C, no CUDA)
CPU_SOURCE = "mpdp_cpu.c"
CPU_LIB_PATH = os.path.join(OUT_DIR, "libmpdp_cpu.so")
SOURCES = ["mpdp_kernels.cu", "mpdp_api.cu", "mpdp_noalloc.cu", "mpdp_server.cu", "mpdp_xd.cu",
           "mpdp_heuristic.cu", "mpdp_mlp.cu", "mpdp_probe.cu", "mpdp_persist.cu"]
# per-file extra nvcc flags (none at present)
EXTRA_FLAGS = {}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-fno-fast-math", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "mpdp.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(path: str = LIB_PATH) -> bool:
    if not os.path.exists(path):
        return False
    t = os.path.getmtime(path)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build_cpu(force: bool = False) -> str:
    """libmpdp_cpu.so: gcc, C11 + pthreads, no FMA contraction."""
    if not force and up_to_date(CPU_LIB_PATH):
        return CPU_LIB_PATH
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = CPU_LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-pthread", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-o", tmp, os.path.join(CSRC, CPU_SOURCE), "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed for {CPU_SOURCE}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, CPU_LIB_PATH)
    return CPU_LIB_PATH


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    build_cpu(force)
    if not force and up_to_date():
        return LIB_PATH
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *EXTRA_FLAGS.get(src, []), *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_info:
            print(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, ptxas_info="-v" in sys.argv))
