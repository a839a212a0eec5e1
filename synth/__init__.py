"""Seeded synthetic particle sets (shared input generator).

This package only produces inputs; it contains none of the short-range force,
sort, rung or kick arithmetic.  Both the CUDA path's tests/benchmark and the
CPU oracle draw their inputs from here.  See ``synth.c`` for the recipe.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .workloads import WORKLOADS, Workload, workload  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into _synth.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, u64, d, p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
            lib.synth_positions.argtypes = [i64, u64, d, i64, d, d, d, p, p, p]
            lib.synth_positions.restype = i64
            lib.synth_uniform.argtypes = [i64, u64, u64, d, d, p]
            lib.synth_uniform.restype = None
            lib.synth_uniform_int8.argtypes = [i64, u64, u64, ctypes.c_int, p]
            lib.synth_uniform_int8.restype = None
            _lib = lib
    return _lib


def positions(n: int, seed: int, frac_uniform: float, n_spheres: int, b_lo: float, b_hi: float,
              r_max: float = 0.25, out: np.ndarray | None = None) -> np.ndarray:
    """(3, n) float64 positions in [0, 1): uniform part plus Plummer spheres."""
    lib = _load()
    pos = np.empty((3, n), dtype=np.float64) if out is None else out
    assert pos.shape == (3, n) and pos.dtype == np.float64 and pos.flags.c_contiguous
    lib.synth_positions(n, seed, frac_uniform, n_spheres, b_lo, b_hi, r_max,
                        pos[0].ctypes.data, pos[1].ctypes.data, pos[2].ctypes.data)
    return pos


def uniform(n: int, seed: int, stream_base: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n float64 values uniform in [lo, hi) (independent per-element streams)."""
    out = np.empty(n, dtype=np.float64)
    _load().synth_uniform(n, seed, stream_base, lo, hi, out.ctypes.data)
    return out


def uniform_int8(n: int, seed: int, stream_base: int, m: int) -> np.ndarray:
    """n int8 values uniform in [0, m)."""
    out = np.empty(n, dtype=np.int8)
    _load().synth_uniform_int8(n, seed, stream_base, m, out.ctypes.data)
    return out


def workload_positions(w: "Workload", out: np.ndarray | None = None) -> np.ndarray:
    return positions(w.n, w.seed, w.frac_uniform, w.n_spheres, w.b_lo, w.b_hi, out=out)
