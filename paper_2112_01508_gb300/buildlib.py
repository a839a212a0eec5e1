"""Build the CUDA libraries (sm_103a) in-tree.

``build()`` compiles every ``csrc/*.cu`` translation unit with nvcc in
parallel and links ``libp3m_sr.so`` (short-range path) next to this file, and
``csrc/pm/*.cu`` into ``libp3m_pm.so`` (long-range mesh path, linked against
cuFFT).  Objects go to ``_build/`` (git-ignored).  Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libp3m_sr.so")
LIB_PM = os.path.join(HERE, "libp3m_pm.so")
CUDA_LIB = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(shutil.which("nvcc") or
                                                                         "/usr/local/cuda/bin/nvcc"))), "lib64")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                     "-I" + os.path.join(HERE, "..", "include")]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return cand


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    hs += glob.glob(os.path.join(HERE, "..", "include", "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _compile(src: str, obj: str, extra: list[str]) -> None:
    cmd = [_nvcc()] + NVCC_FLAGS + extra + ["-c", src, "-o", obj + ".tmp"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{res.stdout}\n{res.stderr}")
    os.replace(obj + ".tmp", obj)


def _build_one(srcs: list[str], lib: str, link_extra: list[str], force: bool, extra: list[str]) -> None:
    os.makedirs(BUILD, exist_ok=True)
    hdr_t = _headers_mtime()
    jobs = []
    objs = []
    for src in srcs:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_t):
            jobs.append((src, obj))
    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            futs = [ex.submit(_compile, s, o, extra) for s, o in jobs]
            for f in futs:
                f.result()
    if jobs or not os.path.exists(lib):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"] + link_extra
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    """Compile csrc/*.cu and csrc/pm/*.cu for sm_103a and link libp3m_sr.so and
    libp3m_pm.so.  Returns the short-range library's path."""
    extra = list(extra_flags or [])
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    pm_srcs = sorted(glob.glob(os.path.join(CSRC, "pm", "*.cu")))
    with concurrent.futures.ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(_build_one, srcs, LIB, [], force, extra)
        b = ex.submit(_build_one, pm_srcs, LIB_PM, ["-L" + CUDA_LIB, "-lcufft", "-Xlinker", "-rpath=" + CUDA_LIB],
                      force, extra)
        a.result()
        b.result()
    if verbose:
        print("built", LIB, "and", LIB_PM)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
