"""ctypes binding of the C ABI in include/p3m_sr.h (argument marshalling only).

Each ``p3m_sr_*`` function here has the name and argument order of the C entry
point and returns its integer status.  The library must have been built
(``paper_2112_01508_gb300.buildlib.build()``); loading fails loudly otherwise --
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .buildlib import LIB

P3M_OK = 0
P3M_ERR_INVALID = 1
P3M_ERR_TOO_FEW_TILES = 2
P3M_ERR_OOM = 3
P3M_ERR_CUDA = 4
P3M_ERR_TIMEOUT = 5
P3M_ERR_NONFINITE = 6
P3M_ERR_STATE = 7

STATUS_NAMES = {
    0: "P3M_OK", 1: "P3M_ERR_INVALID", 2: "P3M_ERR_TOO_FEW_TILES", 3: "P3M_ERR_OOM", 4: "P3M_ERR_CUDA",
    5: "P3M_ERR_TIMEOUT", 6: "P3M_ERR_NONFINITE", 7: "P3M_ERR_STATE",
}

SOFTENING = {"none": 0, "plummer": 1, "bspline": 2}

# Every symbol declared in include/p3m_sr.h.
EXPORTS = (
    "p3m_sr_create", "p3m_sr_destroy", "p3m_sr_last_error", "p3m_sr_sync", "p3m_sr_stats", "p3m_sr_sort",
    "p3m_sr_build_pairs", "p3m_sr_forces", "p3m_sr_assign_rungs", "p3m_sr_kick", "p3m_sr_drift", "p3m_sr_vjp",
    "p3m_sr_permute", "p3m_sr_unpermute", "p3m_sr_forces_noalloc", "p3m_sr_forces_tabulated",
    "p3m_sr_rung_kick", "p3m_sr_set_subtiles", "p3m_sr_set_symmetric", "p3m_sr_kick_drift",
    "p3m_sr_set_count", "p3m_sr_tile_offsets", "p3m_sr_sort_into", "p3m_sr_rung_kick_drift",
)


class P3MParams(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("box", ctypes.c_double),
        ("x_s", ctypes.c_double),
        ("x_r", ctypes.c_double),
        ("G_m", ctypes.c_double),
        ("softening", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("n_sub", ctypes.c_int * 3),
        ("n_rung", ctypes.c_int),
    ]


class P3MStats(ctypes.Structure):
    _fields_ = [
        ("n_tile", ctypes.c_int),
        ("n_sub", ctypes.c_int * 3),
        ("n_subtiles", ctypes.c_int64),
        ("n_active", ctypes.c_int64),
        ("n_chunks", ctypes.c_int64),
        ("pairs_last", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("force_kernel_ms", ctypes.c_double),
        ("vjp_kernel_ms", ctypes.c_double),
    ]


class P3MError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return LIB


def load() -> ctypes.CDLL:
    """Load libp3m_sr.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB):
            raise ImportError(
                f"{LIB} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB)
        p, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.p3m_sr_create.argtypes = [ctypes.POINTER(P3MParams), p, ctypes.POINTER(p)]
        L.p3m_sr_create.restype = i
        L.p3m_sr_destroy.argtypes = [p]
        L.p3m_sr_destroy.restype = None
        L.p3m_sr_last_error.argtypes = [p]
        L.p3m_sr_last_error.restype = ctypes.c_char_p
        L.p3m_sr_sync.argtypes = [p]
        L.p3m_sr_sync.restype = i
        L.p3m_sr_stats.argtypes = [p, ctypes.POINTER(P3MStats)]
        L.p3m_sr_stats.restype = i
        L.p3m_sr_sort.argtypes = [p, p, ctypes.POINTER(p), ctypes.POINTER(i), i, p, p]
        L.p3m_sr_sort.restype = i
        L.p3m_sr_build_pairs.argtypes = [p, p, i]
        L.p3m_sr_build_pairs.restype = i
        L.p3m_sr_forces.argtypes = [p, p, i, p]
        L.p3m_sr_forces.restype = i
        L.p3m_sr_assign_rungs.argtypes = [p, p, i, d, d, d, p]
        L.p3m_sr_assign_rungs.restype = i
        L.p3m_sr_kick.argtypes = [p, p, i, p, i, p, i, ctypes.POINTER(d)]
        L.p3m_sr_kick.restype = i
        L.p3m_sr_drift.argtypes = [p, p, p, i, d]
        L.p3m_sr_drift.restype = i
        L.p3m_sr_kick_drift.argtypes = [p, p, p, i, p, i, p, d, d, d, ctypes.POINTER(d), d]
        L.p3m_sr_kick_drift.restype = i
        L.p3m_sr_vjp.argtypes = [p, p, i, p, p]
        L.p3m_sr_vjp.restype = i
        L.p3m_sr_permute.argtypes = [p, p, p, i, i]
        L.p3m_sr_permute.restype = i
        L.p3m_sr_unpermute.argtypes = [p, p, p, i, i]
        L.p3m_sr_unpermute.restype = i
        L.p3m_sr_forces_noalloc.argtypes = [ctypes.POINTER(P3MParams), p, p, p]
        L.p3m_sr_forces_noalloc.restype = i
        L.p3m_sr_forces_tabulated.argtypes = [p, p, i, p]
        L.p3m_sr_forces_tabulated.restype = i
        L.p3m_sr_rung_kick.argtypes = [p, p, i, p, i, p, p, i, ctypes.c_longlong, d, d, d, i]
        L.p3m_sr_rung_kick.restype = i
        L.p3m_sr_rung_kick_drift.argtypes = [p, p, i, p, i, p, p, i, ctypes.c_longlong, d, d, d, p, d]
        L.p3m_sr_rung_kick_drift.restype = i
        L.p3m_sr_set_subtiles.argtypes = [p, ctypes.POINTER(i)]
        L.p3m_sr_set_subtiles.restype = i
        L.p3m_sr_set_symmetric.argtypes = [p, i]
        L.p3m_sr_set_symmetric.restype = i
        L.p3m_sr_sort_into.argtypes = [p, p, p, ctypes.POINTER(p), ctypes.POINTER(p), ctypes.POINTER(i), i, p, p]
        L.p3m_sr_sort_into.restype = i
        L.p3m_sr_set_count.argtypes = [p, ctypes.c_int64]
        L.p3m_sr_set_count.restype = i
        L.p3m_sr_tile_offsets.argtypes = [p, p]
        L.p3m_sr_tile_offsets.restype = i
        _lib = L
        return L


# ---- thin wrappers with the C names ------------------------------------------

def p3m_sr_create(params: P3MParams, cuda_stream: int):
    ctx = ctypes.c_void_p()
    st = load().p3m_sr_create(ctypes.byref(params), ctypes.c_void_p(cuda_stream), ctypes.byref(ctx))
    return st, ctx


def p3m_sr_destroy(ctx) -> None:
    load().p3m_sr_destroy(ctx)


def p3m_sr_last_error(ctx) -> str:
    return load().p3m_sr_last_error(ctx).decode(errors="replace")


def p3m_sr_sync(ctx) -> int:
    return load().p3m_sr_sync(ctx)


def p3m_sr_stats(ctx):
    out = P3MStats()
    st = load().p3m_sr_stats(ctx, ctypes.byref(out))
    return st, out


def p3m_sr_set_subtiles(ctx, n_sub) -> int:
    arr = (ctypes.c_int * 3)(*[int(v) for v in n_sub])
    return load().p3m_sr_set_subtiles(ctx, arr)


def p3m_sr_set_symmetric(ctx, enable: bool) -> int:
    return load().p3m_sr_set_symmetric(ctx, 1 if enable else 0)


def p3m_sr_sort(ctx, pos_ptr: int, carry_ptrs, carry_bytes, perm_out_ptr, subtile_id_out_ptr) -> int:
    n = len(carry_ptrs)
    arr = (ctypes.c_void_p * max(n, 1))(*[ctypes.c_void_p(c) for c in carry_ptrs])
    nb = (ctypes.c_int * max(n, 1))(*list(carry_bytes))
    return load().p3m_sr_sort(ctx, ctypes.c_void_p(pos_ptr), arr if n else None, nb if n else None, n,
                              ctypes.c_void_p(perm_out_ptr or 0), ctypes.c_void_p(subtile_id_out_ptr or 0))


def p3m_sr_build_pairs(ctx, rung_ptr, rung_min: int) -> int:
    return load().p3m_sr_build_pairs(ctx, ctypes.c_void_p(rung_ptr or 0), int(rung_min))


def p3m_sr_forces(ctx, pos_ptr: int, precision: int, acc_ptr: int) -> int:
    return load().p3m_sr_forces(ctx, ctypes.c_void_p(pos_ptr), int(precision), ctypes.c_void_p(acc_ptr))


def p3m_sr_assign_rungs(ctx, acc_ptr: int, acc_precision: int, dt: float, eta: float, eps: float, rung_ptr: int) -> int:
    return load().p3m_sr_assign_rungs(ctx, ctypes.c_void_p(acc_ptr), int(acc_precision), float(dt), float(eta),
                                      float(eps), ctypes.c_void_p(rung_ptr))


def p3m_sr_kick(ctx, mom_ptr, mom_precision, acc_ptr, acc_precision, rung_ptr, rung_min, kick_factor) -> int:
    kf = (ctypes.c_double * len(kick_factor))(*[float(k) for k in kick_factor])
    return load().p3m_sr_kick(ctx, ctypes.c_void_p(mom_ptr), int(mom_precision), ctypes.c_void_p(acc_ptr),
                              int(acc_precision), ctypes.c_void_p(rung_ptr or 0), int(rung_min), kf)


def p3m_sr_drift(ctx, pos_ptr, mom_ptr, mom_precision, factor) -> int:
    return load().p3m_sr_drift(ctx, ctypes.c_void_p(pos_ptr), ctypes.c_void_p(mom_ptr), int(mom_precision),
                               float(factor))


def p3m_sr_kick_drift(ctx, pos_ptr, mom_ptr, mom_precision, acc_ptr, acc_precision, rung_ptr, dt, eta, eps,
                      kick_factor, drift_factor) -> int:
    kf = (ctypes.c_double * len(kick_factor))(*[float(k) for k in kick_factor])
    return load().p3m_sr_kick_drift(ctx, ctypes.c_void_p(pos_ptr), ctypes.c_void_p(mom_ptr), int(mom_precision),
                                    ctypes.c_void_p(acc_ptr), int(acc_precision), ctypes.c_void_p(rung_ptr),
                                    float(dt), float(eta), float(eps), kf, float(drift_factor))


def p3m_sr_vjp(ctx, pos_ptr, precision, acc_bar_ptr, pos_bar_ptr) -> int:
    return load().p3m_sr_vjp(ctx, ctypes.c_void_p(pos_ptr), int(precision), ctypes.c_void_p(acc_bar_ptr),
                             ctypes.c_void_p(pos_bar_ptr))


def p3m_sr_permute(ctx, src_ptr, dst_ptr, elem_bytes, rows) -> int:
    return load().p3m_sr_permute(ctx, ctypes.c_void_p(src_ptr), ctypes.c_void_p(dst_ptr), int(elem_bytes), int(rows))


def p3m_sr_unpermute(ctx, src_ptr, dst_ptr, elem_bytes, rows) -> int:
    return load().p3m_sr_unpermute(ctx, ctypes.c_void_p(src_ptr), ctypes.c_void_p(dst_ptr), int(elem_bytes),
                                   int(rows))


def p3m_sr_forces_tabulated(ctx, pos_ptr, table_bits, acc_ptr) -> int:
    return load().p3m_sr_forces_tabulated(ctx, ctypes.c_void_p(pos_ptr), int(table_bits), ctypes.c_void_p(acc_ptr))


def p3m_sr_rung_kick(ctx, mom_ptr, mom_precision, acc_ptr, acc_precision, rung_ptr, state_ptr, rung_min, substep,
                     dt, eta, eps, synchronize) -> int:
    return load().p3m_sr_rung_kick(ctx, ctypes.c_void_p(mom_ptr), int(mom_precision), ctypes.c_void_p(acc_ptr),
                                   int(acc_precision), ctypes.c_void_p(rung_ptr), ctypes.c_void_p(state_ptr),
                                   int(rung_min), int(substep), float(dt), float(eta), float(eps), int(synchronize))


# ---- the long-range mesh library (include/p3m_pm.h) -----------------------------

from .buildlib import LIB_PM  # noqa: E402

# Every symbol declared in include/p3m_pm.h.
PM_EXPORTS = (
    "p3m_pm_create", "p3m_pm_destroy", "p3m_pm_last_error", "p3m_pm_sync", "p3m_pm_stats", "p3m_pm_accel",
    "p3m_pm_assign", "p3m_pm_potential",
)


class PMParams(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("box", ctypes.c_double),
        ("n_phi", ctypes.c_int),
        ("x_s", ctypes.c_double),
        ("G_m", ctypes.c_double),
        ("p_i", ctypes.c_int),
        ("p_d", ctypes.c_int),
        ("precision", ctypes.c_int),
    ]


class PMStats(ctypes.Structure):
    _fields_ = [
        ("n_phi", ctypes.c_int),
        ("mesh_bytes", ctypes.c_int64),
        ("fft_work_bytes", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("assign_ms", ctypes.c_double),
        ("fft_ms", ctypes.c_double),
        ("kernel_ms", ctypes.c_double),
        ("ifft_ms", ctypes.c_double),
        ("interp_ms", ctypes.c_double),
    ]


_pm = None


def pm_lib_path() -> str:
    return LIB_PM


def load_pm() -> ctypes.CDLL:
    """Load libp3m_pm.so; raises if it has not been built."""
    global _pm
    with _lock:
        if _pm is not None:
            return _pm
        if not os.path.exists(LIB_PM):
            raise ImportError(
                f"{LIB_PM} is missing: build the CUDA libraries first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PM)
        p, i = ctypes.c_void_p, ctypes.c_int
        L.p3m_pm_create.argtypes = [ctypes.POINTER(PMParams), p, ctypes.POINTER(p)]
        L.p3m_pm_create.restype = i
        L.p3m_pm_destroy.argtypes = [p]
        L.p3m_pm_destroy.restype = None
        L.p3m_pm_last_error.argtypes = [p]
        L.p3m_pm_last_error.restype = ctypes.c_char_p
        L.p3m_pm_sync.argtypes = [p]
        L.p3m_pm_sync.restype = i
        L.p3m_pm_stats.argtypes = [p, ctypes.POINTER(PMStats)]
        L.p3m_pm_stats.restype = i
        L.p3m_pm_accel.argtypes = [p, p, p, i]
        L.p3m_pm_accel.restype = i
        L.p3m_pm_assign.argtypes = [p, p, p]
        L.p3m_pm_assign.restype = i
        L.p3m_pm_potential.argtypes = [p, p]
        L.p3m_pm_potential.restype = i
        _pm = L
        return L


def p3m_pm_create(params: PMParams, cuda_stream: int):
    ctx = ctypes.c_void_p()
    st = load_pm().p3m_pm_create(ctypes.byref(params), ctypes.c_void_p(cuda_stream), ctypes.byref(ctx))
    return st, ctx


def p3m_pm_destroy(ctx) -> None:
    load_pm().p3m_pm_destroy(ctx)


def p3m_pm_last_error(ctx) -> str:
    return load_pm().p3m_pm_last_error(ctx).decode(errors="replace")


def p3m_pm_sync(ctx) -> int:
    return load_pm().p3m_pm_sync(ctx)


def p3m_pm_stats(ctx):
    out = PMStats()
    st = load_pm().p3m_pm_stats(ctx, ctypes.byref(out))
    return st, out


def p3m_pm_accel(ctx, pos_ptr: int, acc_ptr: int, accumulate: int) -> int:
    return load_pm().p3m_pm_accel(ctx, ctypes.c_void_p(pos_ptr), ctypes.c_void_p(acc_ptr), int(accumulate))


def p3m_pm_assign(ctx, pos_ptr: int, rho_ptr: int) -> int:
    return load_pm().p3m_pm_assign(ctx, ctypes.c_void_p(pos_ptr), ctypes.c_void_p(rho_ptr))


def p3m_pm_potential(ctx, phi_ptr: int) -> int:
    return load_pm().p3m_pm_potential(ctx, ctypes.c_void_p(phi_ptr))


def p3m_sr_set_count(ctx, n) -> int:
    return load().p3m_sr_set_count(ctx, int(n))


def p3m_sr_tile_offsets(ctx, out_ptr) -> int:
    return load().p3m_sr_tile_offsets(ctx, ctypes.c_void_p(out_ptr))


def p3m_sr_sort_into(ctx, pos_in, pos_out, carry_in, carry_out, carry_bytes, perm_ptr, ids_ptr) -> int:
    k = len(carry_out)
    ci = (ctypes.c_void_p * max(k, 1))(*[ctypes.c_void_p(x) for x in carry_in])
    co = (ctypes.c_void_p * max(k, 1))(*[ctypes.c_void_p(x) for x in carry_out])
    cb = (ctypes.c_int * max(k, 1))(*carry_bytes)
    return load().p3m_sr_sort_into(ctx, ctypes.c_void_p(pos_in), ctypes.c_void_p(pos_out), ci, co, cb, k,
                                   ctypes.c_void_p(perm_ptr or 0), ctypes.c_void_p(ids_ptr or 0))


def p3m_sr_rung_kick_drift(ctx, mom_ptr, mom_precision, acc_ptr, acc_precision, rung_ptr, state_ptr, rung_min,
                           substep, dt, eta, eps, pos_ptr, drift_factor) -> int:
    return load().p3m_sr_rung_kick_drift(ctx, ctypes.c_void_p(mom_ptr), int(mom_precision), ctypes.c_void_p(acc_ptr),
                                         int(acc_precision), ctypes.c_void_p(rung_ptr), ctypes.c_void_p(state_ptr),
                                         int(rung_min), int(substep), float(dt), float(eta), float(eps),
                                         ctypes.c_void_p(pos_ptr), float(drift_factor))
