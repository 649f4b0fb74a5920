"""Build liblbm.so (the CUDA library behind include/lbm.h) for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
paper_2504_09024_gb300/_lib/liblbm.so.  Host code builds identically on
x86_64 and aarch64 (no architecture-specific flags).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
SO = os.path.join(LIBDIR, "liblbm.so")
SOURCES = ["lbm_kernels.cu", "lbm_sweep_tma.cu", "lbm_sweep_tma16.cu", "lbm_api.cu", "lbm_noalloc.cu",
           "surr_mlp.cu", "lbm3d.cu"]
HEADERS = ["lbm_device.cuh", "lbm_internal.h", "lbm_cell.cuh", "lbm_tma.cuh", "lbm_sweep2.cuh",
           "lbm_store16.cuh", "lbm_vec.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "lbm.h"))
    files.append(os.path.join(ROOT, "include", "lbm3.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= _newest_input():
        return SO
    cc = nvcc()
    flags = FLAGS + list(extra_flags or [])
    objs = []

    def compile_one(src):
        obj = os.path.join(LIBDIR, os.path.splitext(src)[0] + f".{os.getpid()}.o")
        cmd = [cc] + ARCH + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = SO + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    for o in objs:
        try:
            os.remove(o)
        except OSError:
            pass
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force=True, verbose=True))


SOURCES_3D = ["lbm3d.cu"]


def source_hash(which: str = "2d") -> str:
    """Hash of the sources of one kernel family, keying profiler records:
    "2d" -- the coupled D2Q9 sweeps, their headers and include/lbm.h;
    "3d" -- the D3Q27 step (lbm3d.cu) and include/lbm3.h."""
    import hashlib
    h = hashlib.sha256()
    if which == "3d":
        for f in SOURCES_3D:
            h.update(open(os.path.join(CSRC, f), "rb").read())
        h.update(open(os.path.join(ROOT, "include", "lbm3.h"), "rb").read())
        return h.hexdigest()[:16]
    for f in sorted([f for f in SOURCES if f not in SOURCES_3D] + HEADERS):
        h.update(open(os.path.join(CSRC, f), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "lbm.h"), "rb").read())
    return h.hexdigest()[:16]
