"""Torch-facing wrapper of the long-range mesh library (include/p3m_pm.h).

``LongRange`` owns a p3m_pm context: an n_phi^3 mesh and its cuFFT plans.
``accel`` returns (or adds onto ``out``) the long-range accelerations of
Eq. p3m_gravity's upper half (Section 2.1.3): particles -> mesh with W_p, FFT,
the deconvolved long-range kernel, inverse FFT, symmetric differences D_pd and
mesh -> particles.  All steps run in the library; this module marshals
arguments only.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import _native as nat


@dataclass
class PMStats:
    n_phi: int
    mesh_bytes: int
    fft_work_bytes: int
    kernel_launches: int
    assign_ms: float
    fft_ms: float
    kernel_ms: float
    ifft_ms: float
    interp_ms: float

    @property
    def total_ms(self) -> float:
        return self.assign_ms + self.fft_ms + self.kernel_ms + self.ifft_ms + self.interp_ms


class LongRange:
    """Long-range P3M (or, with x_s = 0, plain PM) accelerations for ``n`` particles."""

    def __init__(self, n: int, n_phi: int, x_s: float, G_m: float, p_i: int = 2, p_d: int = 4,
                 precision: int = 32, box: float = 1.0, device=None, stream=None):
        nat.load_pm()
        dev = torch.device("cuda") if device is None else torch.device(device)
        if dev.type != "cuda":
            raise ValueError("LongRange needs a CUDA device")
        self.device = dev if dev.index is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        p = nat.PMParams()
        p.n, p.box, p.n_phi, p.x_s, p.G_m = int(n), float(box), int(n_phi), float(x_s), float(G_m)
        p.p_i, p.p_d, p.precision = int(p_i), int(p_d), int(precision)
        self.params = p
        self.n = int(n)
        self.n_phi = int(n_phi)
        self.dtype = torch.float32 if precision == 32 else torch.float64
        with torch.cuda.device(self.device):
            st, ctx = nat.p3m_pm_create(p, self.stream.cuda_stream)
        if st != nat.P3M_OK:
            raise nat.P3MError(st, "p3m_pm_create failed (check parameters / device memory)")
        self._ctx = ctx

    @classmethod
    def from_workload(cls, w, **kw):
        """Mesh of Eq. phi_gridsize_preference (n_phi = 2 cbrt(N)) and x_s = 1.25 L_phi."""
        return cls(w.n, w.n_phi, w.x_s, w.G_m, **kw)

    def close(self):
        if getattr(self, "_ctx", None):
            nat.p3m_pm_destroy(self._ctx)
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
            raise nat.P3MError(st, nat.p3m_pm_last_error(self._ctx))

    def _check_pos(self, pos):
        if pos.dtype != torch.float64 or tuple(pos.shape) != (3, self.n) or not pos.is_contiguous() \
                or pos.device != self.device:
            raise ValueError(f"pos must be a contiguous (3, {self.n}) float64 tensor on {self.device}")

    def accel(self, pos: torch.Tensor, out: torch.Tensor | None = None, accumulate: bool = False) -> torch.Tensor:
        self._check_pos(pos)
        if out is None:
            if accumulate:
                raise ValueError("accumulate needs an output tensor")
            out = torch.empty((3, self.n), dtype=self.dtype, device=self.device)
        if out.dtype != self.dtype or tuple(out.shape) != (3, self.n) or not out.is_contiguous() \
                or out.device != self.device:
            raise ValueError(f"out must be a contiguous (3, {self.n}) {self.dtype} tensor on {self.device}")
        self._raise(nat.p3m_pm_accel(self._ctx, pos.data_ptr(), out.data_ptr(), int(accumulate)))
        return out

    def assign(self, pos: torch.Tensor) -> torch.Tensor:
        """rho_m = sum_j W_p((x_m - x_j)/L_phi), dense (n_phi, n_phi, n_phi)."""
        self._check_pos(pos)
        rho = torch.empty((self.n_phi,) * 3, dtype=self.dtype, device=self.device)
        self._raise(nat.p3m_pm_assign(self._ctx, pos.data_ptr(), rho.data_ptr()))
        return rho

    def potential(self) -> torch.Tensor:
        """(4 pi G m / L_phi^4) F^-1{G(k) F rho} of the last accel call, dense (n_phi,)*3."""
        phi = torch.empty((self.n_phi,) * 3, dtype=self.dtype, device=self.device)
        self._raise(nat.p3m_pm_potential(self._ctx, phi.data_ptr()))
        return phi

    def sync(self):
        self._raise(nat.p3m_pm_sync(self._ctx))

    def stats(self) -> PMStats:
        st, s = nat.p3m_pm_stats(self._ctx)
        self._raise(st)
        return PMStats(s.n_phi, s.mesh_bytes, s.fft_work_bytes, s.kernel_launches, s.assign_ms, s.fft_ms,
                       s.kernel_ms, s.ifft_ms, s.interp_ms)
