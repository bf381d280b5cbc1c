"""Build libtsfde.so (CUDA for sm_103a) in-tree with nvcc.

Each translation unit under csrc/ is compiled in parallel to an object file,
then the objects are linked into paper_2507_02809_gb300/lib/libtsfde.so.
Objects are rebuilt when the source or any header is newer.  The mixed-length
persistent kernel (fsub_mix*.cu) is relocatable device code: its per-length
bodies are compiled with at most 128 registers per thread and joined to the
kernel that calls them by a device-link step.
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
LIBDIR = os.path.join(HERE, "lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIBNAME = "libtsfde.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtsfde")


def lib_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def _headers_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    paths.append(os.path.join(ROOT, "include", "tsfde.h"))
    return max(os.path.getmtime(p) for p in paths)


def _extra_flags(name: str) -> list:
    if name.startswith("fsub_mix_"):
        return ["-rdc=true", "-maxrregcount=128"]
    if name.startswith("fsub_mix"):
        return ["-rdc=true"]
    return []


def _compile(src: str, obj: str, verbose: bool) -> None:
    cmd = [nvcc()] + ARCH + FLAGS + _extra_flags(os.path.basename(src)) + ["-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, res.stdout, res.stderr))


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OBJDIR, exist_ok=True)
    sources = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    hdr = _headers_mtime()
    jobs = []
    objs = []
    for f in sources:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OBJDIR, f[:-3] + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr):
            jobs.append((src, obj))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(lambda j: _compile(j[0], j[1], verbose), jobs))
    out = lib_path()
    if jobs or not os.path.exists(out):
        rdc = [o for o in objs if os.path.basename(o).startswith("fsub_mix")]
        dlink = os.path.join(OBJDIR, "dlink.o")
        if rdc:
            cmd = [nvcc()] + ARCH + ["-Xcompiler", "-fPIC", "-dlink", "-o", dlink] + rdc
            res = subprocess.run(cmd, capture_output=True, text=True)
            if res.returncode != 0:
                raise RuntimeError("device link failed:\n%s\n%s" % (res.stdout, res.stderr))
        tmp = out + ".tmp"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ([dlink] if rdc else []) + ["-lcudadevrt", "-lcudart"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (res.stdout, res.stderr))
        os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
