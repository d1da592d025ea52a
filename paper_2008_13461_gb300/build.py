"""In-tree build of the CUDA library libpt_gb300.so (sm_103a only).

Each translation unit under csrc/ is compiled by nvcc in parallel, then
linked into a shared library next to this file (lib/libpt_gb300.so).  No
cmake, no torch extension machinery: the library has a plain C ABI
(include/pt.h) and is loaded with ctypes."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(OUT_DIR, "libpt_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["pt_bin.cu", "pt_doublets.cu", "pt_fishbone.cu", "pt_connect.cu", "pt_ntuplets.cu", "pt_fit.cu",
           "pt_fit_grad.cu", "pt_postfit.cu", "pt_vertex.cu", "pt_probe.cu", "pt_abi.cu",
           "pt_noalloc.cu", "pt_timing.cu"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpt_gb300.so")


def _flags(verbose_ptxas: bool):
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")] + ARCH
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "pt.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None) -> str:
    """Compile csrc/*.cu for sm_103a and link lib/libpt_gb300.so; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    objs = [os.path.join(OUT_DIR, s.replace(".cu", ".o")) for s in SOURCES]

    def one(src_obj):
        src, obj = src_obj
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(verbose_ptxas)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(SOURCES), os.cpu_count() or 4)) as ex:
        logs = list(ex.map(one, zip(SOURCES, objs)))
    tmp = LIB + ".tmp"
    r = subprocess.run([cc, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose_ptxas:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose_ptxas=True))
