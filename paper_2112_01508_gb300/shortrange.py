"""Torch-facing wrapper of the C ABI: one ``ShortRange`` object per context.

All arithmetic runs in the library's CUDA kernels; this module only checks
tensor shapes/dtypes/devices and passes raw device pointers.  Tensors are
structure-of-arrays ``(3, n)`` and must be contiguous on the context's device.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _native as nat

_PREC = {torch.float32: 32, torch.float64: 64}


@dataclass
class Stats:
    n_tile: int
    n_sub: tuple
    n_subtiles: int
    n_active: int
    n_chunks: int
    pairs_last: int
    kernel_launches: int
    force_kernel_ms: float
    vjp_kernel_ms: float


def _check(t: torch.Tensor, name: str, dtype=None, shape=None, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if device is not None and t.device != device:
        raise ValueError(f"{name} must be on {device}, got {t.device}")


def _swap_storage(a: torch.Tensor, b: torch.Tensor):
    """Exchange the memory behind two tensors of one shape and dtype (no copy)."""
    sa, sb = a.untyped_storage(), b.untyped_storage()
    oa, ob = a.storage_offset(), b.storage_offset()
    shape, sta, stb = a.shape, a.stride(), b.stride()
    a.set_(sb, ob, shape, stb)
    b.set_(sa, oa, shape, sta)


class ShortRange:
    """Short-range P3M force context for ``n`` particles (see include/p3m_sr.h)."""

    def __init__(self, n: int, x_s: float, x_r: float, G_m: float, softening: str | int = "bspline",
                 eps: float = 0.0, n_sub=2, n_rung: int = 8, box: float = 1.0, device=None, stream=None,
                 symmetric: bool = True):
        nat.load()
        dev = torch.device("cuda") if device is None else torch.device(device)
        if dev.type != "cuda":
            raise ValueError("ShortRange needs a CUDA device")
        self.device = dev if dev.index is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ns = (n_sub,) * 3 if isinstance(n_sub, int) else tuple(n_sub)
        soft = nat.SOFTENING[softening] if isinstance(softening, str) else int(softening)
        p = nat.P3MParams()
        p.n, p.box, p.x_s, p.x_r, p.G_m = int(n), float(box), float(x_s), float(x_r), float(G_m)
        p.softening, p.eps, p.n_rung = soft, float(eps), int(n_rung)
        p.n_sub[0], p.n_sub[1], p.n_sub[2] = ns
        self.params = p
        self.n = int(n)
        self.n_rung = int(n_rung)
        self.n_sub = ns
        with torch.cuda.device(self.device):
            st, ctx = nat.p3m_sr_create(p, self.stream.cuda_stream)
        if st != nat.P3M_OK:
            raise nat.P3MError(st, "p3m_sr_create failed (check parameters / device memory)")
        self._ctx = ctx
        self.set_symmetric(symmetric)

    @classmethod
    def from_workload(cls, w, **kw):
        kw.setdefault("softening", "bspline")
        kw.setdefault("eps", w.eps)
        kw.setdefault("n_sub", w.n_sub)
        return cls(w.n, w.x_s, w.x_r, w.G_m, **kw)

    # -- lifetime ---------------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None):
            nat.p3m_sr_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _raise(self, st: int):
        if st != nat.P3M_OK:
            raise nat.P3MError(st, nat.p3m_sr_last_error(self._ctx))

    # -- entry points ------------------------------------------------------------
    def set_symmetric(self, enable: bool):
        """All-active FP32 forces: evaluate each pair once and update both particles
        (True, p3m_sr_set_symmetric) or gather per receiver, bitwise reproducible (False)."""
        self._raise(nat.p3m_sr_set_symmetric(self._ctx, bool(enable)))
        self.symmetric = bool(enable)

    def set_count(self, n: int):
        """Particles of the following calls, at most the count given at creation
        (p3m_sr_set_count; no allocation).  Sort again before the next force call."""
        self._raise(nat.p3m_sr_set_count(self._ctx, int(n)))
        self.n = int(n)

    @property
    def capacity(self) -> int:
        return int(self.params.n)

    def tile_offsets(self, out: torch.Tensor | None = None) -> torch.Tensor:
        """Sorted index of the first particle of every tile of the last sort, and n at the
        end (p3m_sr_tile_offsets): a device tensor of n_t^3 + 1 int32."""
        n_t = self.stats_geometry()[0]
        if out is None:
            out = torch.empty(n_t ** 3 + 1, dtype=torch.int32, device=self.device)
        _check(out, "out", torch.int32, (n_t ** 3 + 1,), self.device)
        self._raise(nat.p3m_sr_tile_offsets(self._ctx, out.data_ptr()))
        return out

    def stats_geometry(self):
        """(n_t, n_sub): tiles per dimension and subtiles per tile, from the parameters."""
        import math
        return int(math.floor(self.params.box / self.params.x_r)), self.n_sub

    def set_subtiles(self, n_sub):
        """Change the subtiles per tile (p3m_sr_set_subtiles); sort again before the next force call."""
        ns = (n_sub,) * 3 if isinstance(n_sub, int) else tuple(int(v) for v in n_sub)
        self._raise(nat.p3m_sr_set_subtiles(self._ctx, ns))
        self.n_sub = ns

    def sort(self, pos: torch.Tensor, carry=(), perm_out: torch.Tensor | None = None,
             subtile_id_out: torch.Tensor | None = None, scratch=None):
        """Sort into tile -> subtile walk order.  Without `scratch`: in place (p3m_sr_sort).
        With `scratch`, a list of tensors like [pos, *carry]: out of place into the scratch
        tensors (p3m_sr_sort_into, no copy back), after which each tensor and its scratch
        exchange their storage, so pos and carry hold the sorted data as after an
        in-place sort and the scratch tensors hold the old data."""
        if scratch is not None:
            arrays = [pos, *carry]
            if len(scratch) != len(arrays):
                raise ValueError("scratch must hold one tensor per array of [pos, *carry]")
            self.sort_into(pos, scratch[0], carry, scratch[1:], perm_out, subtile_id_out)
            for a, b in zip(arrays, scratch):
                _swap_storage(a, b)
            return
        _check(pos, "pos", torch.float64, (3, self.n), self.device)
        ptrs, nbytes = [], []
        for c in carry:
            _check(c, "carry", device=self.device)
            if c.numel() % self.n != 0 and self.n > 0:
                raise ValueError("carry tensors must hold n elements (any trailing shape)")
            # a (3, n) SoA tensor is carried as three arrays of n elements
            if c.dim() == 2 and c.shape[0] == 3 and c.shape[1] == self.n and self.n > 0:
                es = c.element_size()
                for d in range(3):
                    ptrs.append(c[d].data_ptr())
                    nbytes.append(es)
            else:
                ptrs.append(c.data_ptr())
                nbytes.append(c.element_size() * (c.numel() // max(self.n, 1)))
        if perm_out is not None:
            _check(perm_out, "perm_out", torch.int32, (self.n,), self.device)
        if subtile_id_out is not None:
            _check(subtile_id_out, "subtile_id_out", torch.int32, (self.n,), self.device)
        st = nat.p3m_sr_sort(self._ctx, pos.data_ptr(), ptrs, nbytes,
                             perm_out.data_ptr() if perm_out is not None else 0,
                             subtile_id_out.data_ptr() if subtile_id_out is not None else 0)
        self._raise(st)

    def _carry_ptrs(self, carry, name):
        ptrs, nbytes = [], []
        for c in carry:
            _check(c, name, device=self.device)
            if c.numel() % max(self.n, 1) != 0 and self.n > 0:
                raise ValueError("carry tensors must hold n elements (any trailing shape)")
            if c.dim() == 2 and c.shape[0] == 3 and c.shape[1] == self.n and self.n > 0:
                es = c.element_size()
                for d in range(3):
                    ptrs.append(c[d].data_ptr())
                    nbytes.append(es)
            else:
                ptrs.append(c.data_ptr())
                nbytes.append(c.element_size() * (c.numel() // max(self.n, 1)))
        return ptrs, nbytes

    def sort_into(self, pos: torch.Tensor, pos_out: torch.Tensor, carry=(), carry_out=(),
                  perm_out: torch.Tensor | None = None, subtile_id_out: torch.Tensor | None = None):
        """Out-of-place sort (p3m_sr_sort_into): pos_out and carry_out receive the sorted
        copies of pos and carry; the inputs are unchanged."""
        _check(pos, "pos", torch.float64, (3, self.n), self.device)
        _check(pos_out, "pos_out", torch.float64, (3, self.n), self.device)
        if len(carry) != len(carry_out):
            raise ValueError("carry and carry_out must pair up")
        for a, b in zip(carry, carry_out):
            if a.dtype != b.dtype or a.shape != b.shape:
                raise ValueError("carry_out must match carry in dtype and shape")
        pin, nb = self._carry_ptrs(carry, "carry")
        pout, _ = self._carry_ptrs(carry_out, "carry_out")
        if perm_out is not None:
            _check(perm_out, "perm_out", torch.int32, (self.n,), self.device)
        if subtile_id_out is not None:
            _check(subtile_id_out, "subtile_id_out", torch.int32, (self.n,), self.device)
        self._raise(nat.p3m_sr_sort_into(self._ctx, pos.data_ptr(), pos_out.data_ptr(), pin, pout, nb,
                                         perm_out.data_ptr() if perm_out is not None else 0,
                                         subtile_id_out.data_ptr() if subtile_id_out is not None else 0))

    def build_pairs(self, rung: torch.Tensor | None = None, rung_min: int = 0):
        if rung is not None:
            _check(rung, "rung", torch.int8, (self.n,), self.device)
        self._raise(nat.p3m_sr_build_pairs(self._ctx, rung.data_ptr() if rung is not None else 0, rung_min))

    def forces(self, pos: torch.Tensor, precision: int = 32, out: torch.Tensor | None = None) -> torch.Tensor:
        _check(pos, "pos", torch.float64, (3, self.n), self.device)
        dt = torch.float32 if precision == 32 else torch.float64
        if out is None:
            out = torch.zeros((3, self.n), dtype=dt, device=self.device)
        _check(out, "out", dt, (3, self.n), self.device)
        self._raise(nat.p3m_sr_forces(self._ctx, pos.data_ptr(), precision, out.data_ptr()))
        return out

    def forces_tabulated(self, pos: torch.Tensor, table_bits: int = 12,
                         out: torch.Tensor | None = None) -> torch.Tensor:
        """FP32 forces with the bracket read from a 2^table_bits NGP table in r^2."""
        _check(pos, "pos", torch.float64, (3, self.n), self.device)
        if out is None:
            out = torch.zeros((3, self.n), dtype=torch.float32, device=self.device)
        _check(out, "out", torch.float32, (3, self.n), self.device)
        self._raise(nat.p3m_sr_forces_tabulated(self._ctx, pos.data_ptr(), table_bits, out.data_ptr()))
        return out

    def assign_rungs(self, acc: torch.Tensor, dt: float, eta: float, eps: float,
                     out: torch.Tensor | None = None) -> torch.Tensor:
        _check(acc, "acc", (torch.float32, torch.float64), (3, self.n), self.device)
        if out is None:
            out = torch.empty(self.n, dtype=torch.int8, device=self.device)
        _check(out, "out", torch.int8, (self.n,), self.device)
        self._raise(nat.p3m_sr_assign_rungs(self._ctx, acc.data_ptr(), _PREC[acc.dtype], dt, eta, eps,
                                            out.data_ptr()))
        return out

    def kick(self, mom: torch.Tensor, acc: torch.Tensor, kick_factor, rung: torch.Tensor | None = None,
             rung_min: int = 0):
        _check(mom, "mom", (torch.float32, torch.float64), (3, self.n), self.device)
        _check(acc, "acc", (torch.float32, torch.float64), (3, self.n), self.device)
        if rung is not None:
            _check(rung, "rung", torch.int8, (self.n,), self.device)
        kf = [float(k) for k in kick_factor]
        if len(kf) < self.n_rung:
            kf = kf + [kf[-1]] * (self.n_rung - len(kf))
        self._raise(nat.p3m_sr_kick(self._ctx, mom.data_ptr(), _PREC[mom.dtype], acc.data_ptr(), _PREC[acc.dtype],
                                    rung.data_ptr() if rung is not None else 0, rung_min, kf))

    def rung_kick(self, mom: torch.Tensor, acc: torch.Tensor, rung: torch.Tensor, kick_state: torch.Tensor,
                  rung_min: int, substep: int, dt: float, eta: float, eps: float, synchronize: bool = False):
        """One kick of the rung-based leapfrog with rung jumps (p3m_sr_rung_kick)."""
        _check(mom, "mom", (torch.float32, torch.float64), (3, self.n), self.device)
        _check(acc, "acc", (torch.float32, torch.float64), (3, self.n), self.device)
        _check(rung, "rung", torch.int8, (self.n,), self.device)
        _check(kick_state, "kick_state", torch.int8, (self.n,), self.device)
        self._raise(nat.p3m_sr_rung_kick(self._ctx, mom.data_ptr(), _PREC[mom.dtype], acc.data_ptr(), _PREC[acc.dtype],
                                         rung.data_ptr(), kick_state.data_ptr(), rung_min, substep, dt, eta, eps,
                                         int(synchronize)))

    def rung_kick_drift(self, mom: torch.Tensor, acc: torch.Tensor, rung: torch.Tensor, kick_state: torch.Tensor,
                        rung_min: int, substep: int, dt: float, eta: float, eps: float, pos: torch.Tensor,
                        drift_factor: float):
        """rung_kick (not synchronising) then drift of every particle, in one pass
        (p3m_sr_rung_kick_drift; bit for bit the two calls)."""
        _check(mom, "mom", (torch.float32, torch.float64), (3, self.n), self.device)
        _check(acc, "acc", (torch.float32, torch.float64), (3, self.n), self.device)
        _check(rung, "rung", torch.int8, (self.n,), self.device)
        _check(kick_state, "kick_state", torch.int8, (self.n,), self.device)
        _check(pos, "pos", torch.float64, (3, self.n), self.device)
        self._raise(nat.p3m_sr_rung_kick_drift(self._ctx, mom.data_ptr(), _PREC[mom.dtype], acc.data_ptr(),
                                               _PREC[acc.dtype], rung.data_ptr(), kick_state.data_ptr(), rung_min,
                                               substep, dt, eta, eps, pos.data_ptr(), drift_factor))

    def drift(self, pos: torch.Tensor, mom: torch.Tensor, factor: float):
        _check(pos, "pos", torch.float64, (3, self.n), self.device)
        _check(mom, "mom", (torch.float32, torch.float64), (3, self.n), self.device)
        self._raise(nat.p3m_sr_drift(self._ctx, pos.data_ptr(), mom.data_ptr(), _PREC[mom.dtype], factor))

    def kick_drift(self, pos: torch.Tensor, mom: torch.Tensor, acc: torch.Tensor, rung_out: torch.Tensor,
                   dt: float, eta: float, eps: float, kick_factor, drift_factor: float):
        """Rungs (Eq. rung), kick and drift in one pass (p3m_sr_kick_drift): the results of
        assign_rungs + kick(rung_min=0) + drift, bit for bit."""
        _check(pos, "pos", torch.float64, (3, self.n), self.device)
        _check(mom, "mom", (torch.float32, torch.float64), (3, self.n), self.device)
        _check(acc, "acc", (torch.float32, torch.float64), (3, self.n), self.device)
        _check(rung_out, "rung_out", torch.int8, (self.n,), self.device)
        kf = [float(k) for k in kick_factor]
        if len(kf) < self.n_rung:
            kf = kf + [kf[-1]] * (self.n_rung - len(kf))
        self._raise(nat.p3m_sr_kick_drift(self._ctx, pos.data_ptr(), mom.data_ptr(), _PREC[mom.dtype],
                                          acc.data_ptr(), _PREC[acc.dtype], rung_out.data_ptr(), dt, eta, eps, kf,
                                          drift_factor))

    def vjp(self, pos: torch.Tensor, acc_bar: torch.Tensor, precision: int | None = None,
            out: torch.Tensor | None = None) -> torch.Tensor:
        _check(pos, "pos", torch.float64, (3, self.n), self.device)
        prec = precision or _PREC[acc_bar.dtype]
        dt = torch.float32 if prec == 32 else torch.float64
        _check(acc_bar, "acc_bar", dt, (3, self.n), self.device)
        if out is None:
            out = torch.empty((3, self.n), dtype=dt, device=self.device)
        _check(out, "out", dt, (3, self.n), self.device)
        self._raise(nat.p3m_sr_vjp(self._ctx, pos.data_ptr(), prec, acc_bar.data_ptr(), out.data_ptr()))
        return out

    def permute(self, src: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Caller order -> order of the last sort (last dimension indexes particles)."""
        return self._perm(src, out, nat.p3m_sr_permute)

    def unpermute(self, src: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Order of the last sort -> caller order."""
        return self._perm(src, out, nat.p3m_sr_unpermute)

    def _perm(self, src, out, fn):
        _check(src, "src", device=self.device)
        if src.shape[-1] != self.n:
            raise ValueError("last dimension must be n")
        if out is None:
            out = torch.empty_like(src)
        _check(out, "out", src.dtype, tuple(src.shape), self.device)
        rows = src.numel() // max(self.n, 1)
        self._raise(fn(self._ctx, src.data_ptr(), out.data_ptr(), src.element_size(), rows))
        return out

    def sync(self):
        self._raise(nat.p3m_sr_sync(self._ctx))

    def stats(self) -> Stats:
        st, s = nat.p3m_sr_stats(self._ctx)
        self._raise(st)
        return Stats(s.n_tile, tuple(s.n_sub), s.n_subtiles, s.n_active, s.n_chunks, s.pairs_last,
                     s.kernel_launches, s.force_kernel_ms, s.vjp_kernel_ms)
