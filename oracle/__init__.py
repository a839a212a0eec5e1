"""CPU oracle for the short-range P3M force -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never calls, links or loads
it.  The C source (``oracle.c``) is a plain FP64 restatement of the paper's
short-range sum (Section 2.1.3, Eq. p3m_gravity), the rung rule (Eq. rung) and
the kick/drift operators (Section 2.2.2).

Parity pins (each checked by a ``-m "not gpu"`` test):
  * bracket B(r) against the gradient of the Ewald short-range potential
    erfc(r/2x_s)/r and Gauss's law for the softening shapes (mpmath);
  * cell-list sum against O(N^2) brute force, and against an explicit sum over
    the 27 nearest periodic images;
  * Newton's third law, permutation and translation invariance;
  * VJP against central finite differences of the oracle's own forward;
  * rungs against the log2/ceil definition; subtile ids against floor().

The long-range (particle-mesh) half of Eq. p3m_gravity is restated in
``oracle/pm.py`` (numpy, FP64) with its own pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

SOFTENING = {"none": 0, "plummer": 1, "bspline": 2}


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so (gcc, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, d, p, i = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
            lib.oracle_bracket.argtypes = [d, d, i, d]
            lib.oracle_bracket.restype = d
            lib.oracle_bracket_dr.argtypes = [d, d, i, d]
            lib.oracle_bracket_dr.restype = d
            common = [d, d, d, d, i, d]
            lib.oracle_sr_accel.argtypes = [i64, p, p, i] + common + [p]
            lib.oracle_sr_accel.restype = i64
            lib.oracle_sr_accel_brute.argtypes = [i64, p, p, i] + common + [p]
            lib.oracle_sr_accel_brute.restype = i64
            lib.oracle_sr_accel_subset.argtypes = [i64, p, i64, p] + common + [p, p]
            lib.oracle_sr_accel_subset.restype = i64
            lib.oracle_sr_vjp.argtypes = [i64, p, p, i] + common + [p, p]
            lib.oracle_sr_vjp.restype = i64
            lib.oracle_subtile_ids.argtypes = [i64, p, i, i, p]
            lib.oracle_subtile_ids.restype = None
            lib.oracle_rungs.argtypes = [i64, p, d, d, d, i, p]
            lib.oracle_rungs.restype = i64
            lib.oracle_kick.argtypes = [i64, p, p, p, i, p]
            lib.oracle_kick.restype = None
            lib.oracle_drift.argtypes = [i64, p, p, d, d]
            lib.oracle_drift.restype = None
            lib.oracle_rung_kick.argtypes = [i64, p, p, p, p, i, ctypes.c_longlong, i, d, d, d, i]
            lib.oracle_rung_kick.restype = i64
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = i
            lib.oracle_set_num_threads.argtypes = [i]
            lib.oracle_set_num_threads.restype = None
            _lib = lib
    return _lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


def _soft(s):
    return SOFTENING[s] if isinstance(s, str) else int(s)


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_num_threads(k: int) -> None:
    """Threads used by the oracle's parallel loops from now on."""
    _load().oracle_set_num_threads(int(k))


def bracket(r, x_s, softening="bspline", eps=0.0):
    """B(r) of Eq. p3m_gravity (without -G m), vectorised over r."""
    lib = _load()
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    return np.array([lib.oracle_bracket(float(v), x_s, _soft(softening), eps) for v in r])


def bracket_dr(r, x_s, softening="bspline", eps=0.0):
    lib = _load()
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    return np.array([lib.oracle_bracket_dr(float(v), x_s, _soft(softening), eps) for v in r])


def _rung_arg(rung):
    if rung is None:
        return None
    return np.ascontiguousarray(rung, dtype=np.int8)


def sr_accel(pos, x_s, x_r, G_m, softening="bspline", eps=0.0, rung=None, rung_min=0, box=1.0,
             out=None, brute=False):
    """Short-range accelerations (3, N) and the interacting-pair count.

    Rows of inactive receivers (rung < rung_min) are left as in ``out``
    (zeros by default)."""
    pos = _f64(pos)
    n = pos.shape[1]
    acc = np.zeros((3, n)) if out is None else out
    rg = _rung_arg(rung)
    fn = _load().oracle_sr_accel_brute if brute else _load().oracle_sr_accel
    pairs = fn(n, _ptr(pos), _ptr(rg), rung_min, box, x_s, x_r, G_m, _soft(softening), eps, _ptr(acc))
    if pairs < 0:
        raise ValueError("oracle: fewer than 3 cells per dimension (x_r too large for the box)")
    return acc, int(pairs)


def sr_accel_subset(pos, receivers, x_s, x_r, G_m, softening="bspline", eps=0.0, box=1.0):
    """Accelerations (3, n_sub) of the listed receivers and per-receiver pair counts."""
    pos = _f64(pos)
    n = pos.shape[1]
    recv = np.ascontiguousarray(receivers, dtype=np.int64)
    acc = np.zeros((3, len(recv)))
    pairs = np.zeros(len(recv), dtype=np.int64)
    tot = _load().oracle_sr_accel_subset(n, _ptr(pos), len(recv), _ptr(recv), box, x_s, x_r, G_m,
                                         _soft(softening), eps, _ptr(acc), _ptr(pairs))
    if tot < 0:
        raise ValueError("oracle: bad geometry")
    return acc, pairs


def sr_vjp(pos, abar, x_s, x_r, G_m, softening="bspline", eps=0.0, rung=None, rung_min=0, box=1.0):
    """xbar = (d a / d x)^T abar over all particles, (3, N)."""
    pos = _f64(pos)
    abar = _f64(abar)
    n = pos.shape[1]
    xbar = np.zeros((3, n))
    rg = _rung_arg(rung)
    tot = _load().oracle_sr_vjp(n, _ptr(pos), _ptr(rg), rung_min, box, x_s, x_r, G_m, _soft(softening),
                                eps, _ptr(abar), _ptr(xbar))
    if tot < 0:
        raise ValueError("oracle: bad geometry")
    return xbar


def subtile_ids(pos, n_tile, n_sub):
    pos = _f64(pos)
    n = pos.shape[1]
    ids = np.empty(n, dtype=np.int32)
    _load().oracle_subtile_ids(n, _ptr(pos), n_tile, n_sub, _ptr(ids))
    return ids


def rungs(acc, dt, eta, eps, n_rung=8):
    acc = _f64(acc)
    n = acc.shape[1]
    out = np.empty(n, dtype=np.int8)
    bad = _load().oracle_rungs(n, _ptr(acc), dt, eta, eps, n_rung, _ptr(out))
    return out, int(bad)


def kick(mom, acc, kick_factor, rung=None, rung_min=0):
    mom = _f64(mom).copy()
    acc = _f64(acc)
    kf = np.ascontiguousarray(kick_factor, dtype=np.float64)
    _load().oracle_kick(mom.shape[1], _ptr(mom), _ptr(acc), _ptr(_rung_arg(rung)), rung_min, _ptr(kf))
    return mom


def drift(pos, mom, factor, box=1.0):
    pos = _f64(pos).copy()
    mom = _f64(mom)
    _load().oracle_drift(pos.shape[1], _ptr(pos), _ptr(mom), factor, box)
    return pos


def rung_kick(mom, acc, rung, state, rung_min, substep, n_rung, dt, eta, eps, sync=False):
    """One kick of the rung-based leapfrog; mom, rung, state are updated in place."""
    assert mom.dtype == np.float64 and mom.flags.c_contiguous
    assert rung.dtype == np.int8 and state.dtype == np.int8
    acc = _f64(acc)
    return _load().oracle_rung_kick(mom.shape[1], _ptr(mom), _ptr(acc), _ptr(rung), _ptr(state), int(rung_min),
                                    int(substep), int(n_rung), float(dt), float(eta), float(eps), int(bool(sync)))


def rung_leapfrog(pos, mom, x_s, x_r, G_m, softening, eps, dt, eta, n_rung, n_steps, period=None, box=1.0,
                  n_phi=None, p_i=2, p_d=4):
    """The rung-based KDK of Section 2.2.2 (the time-stepping figure) over
    n_steps global steps of size dt, synchronised after every `period` steps
    (default: once, at the end).

    A period starts synchronised: rungs from Eq. rung on the forces of all
    particles (the fake kick of the first period; the synchronising kick, in
    which every particle is a receiver, for later ones), then the half kicks
    dt/2^(l+1) per rung.  Each global step is 2^(n_rung-1) substeps of a drift
    dt/2^(n_rung-1) followed by the kick of the rungs due at that time.
    With n_phi given, the long-range mesh force (oracle.pm, orders p_i, p_d) kicks
    every particle whenever rung 0 is kicked: dt/2 at the start of a period, dt at
    the end of each global step (dt/2 at a synchronisation), after the short-range
    kick.  Returns (pos, mom, rung, state, rung_history)."""
    from . import pm as _pm
    pos = _f64(pos).copy()
    mom = _f64(mom).copy()
    period = n_steps if period is None else period
    n = pos.shape[1]
    acc, _ = sr_accel(pos, x_s, x_r, G_m, softening, eps, box=box)
    sub = 2 ** (n_rung - 1)
    history = []
    for step in range(n_steps):
        if step % period == 0:
            rung, _ = rungs(acc, dt, eta, eps, n_rung)
            state = np.zeros(n, dtype=np.int8)
            mom = kick(mom, acc, [dt / 2.0 ** (l + 1) for l in range(n_rung)], rung=rung, rung_min=0)
            if n_phi:
                mom = kick(mom, _pm.lr_accel(pos, n_phi, x_s, G_m, p_i, p_d, box), [dt / 2.0])
            k = 0  # substeps since the synchronisation
        last_of_period = (step + 1) % period == 0 or step == n_steps - 1
        for s in range(1, sub + 1):
            k += 1
            pos = drift(pos, mom, dt / sub, box)
            tz = 0
            while tz < n_rung - 1 and (k >> tz) & 1 == 0:
                tz += 1
            lmin = n_rung - 1 - tz
            acc, _ = sr_accel(pos, x_s, x_r, G_m, softening, eps, rung=rung, rung_min=lmin, box=box, out=acc)
            rung_kick(mom, acc, rung, state, lmin, k, n_rung, dt, eta, eps, last_of_period and s == sub)
            if n_phi and s == sub:
                kf = dt / 2.0 if last_of_period else dt
                mom = kick(mom, _pm.lr_accel(pos, n_phi, x_s, G_m, p_i, p_d, box), [kf])
            history.append(rung.copy())
    return pos, mom, rung, state, history
