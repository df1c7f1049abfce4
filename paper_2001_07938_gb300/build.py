"""Build liblilac.so (the C-ABI library of include/lilac.h) for sm_103a.

Each translation unit in csrc/ is compiled by nvcc in parallel, then linked
into one shared library under _build/ (in-tree, git-ignored).  Run
``python -m paper_2001_07938_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liblilac.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the library is CUDA-only and has no CPU build")
    return cand


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers_mtime() -> float:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(HERE, "..", "include", "lilac.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None,
          extra_flags=(), build_dir: str | None = None) -> str:
    """Compile and link; `extra_flags` (e.g. -D tile-shape overrides) and
    `build_dir` allow side-by-side builds of other configurations."""
    nvcc = _nvcc()
    bdir = build_dir or BUILD_DIR
    lib = os.path.join(bdir, "liblilac.so")
    os.makedirs(bdir, exist_ok=True)
    srcs = sources()
    hdr_t = _headers_mtime()
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
             "--expt-relaxed-constexpr", "-Xcudafe", "--diag_suppress=177", *extra_flags]
    if verbose_ptxas:
        flags += ["-Xptxas", "-v"]

    def obj_of(src):
        return os.path.join(bdir, os.path.basename(src)[:-3] + ".o")

    def compile_one(src):
        obj = obj_of(src)
        if (not force and os.path.exists(obj) and os.path.getmtime(obj) >= os.path.getmtime(src)
                and os.path.getmtime(obj) >= hdr_t):
            return obj, ""
        cmd = [nvcc, *flags, "-c", src, "-o", obj]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{p.stderr}")
        return obj, p.stderr

    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    logs = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = []
        for obj, log in ex.map(compile_one, srcs):
            objs.append(obj)
            if log:
                logs.append(log)
    if (force or not os.path.exists(lib)
            or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs)):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"link failed:\n{p.stderr}")
        os.replace(tmp, lib)
    if verbose_ptxas:
        sys.stderr.write("\n".join(logs))
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
