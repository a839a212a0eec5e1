"""The allocation-free entry point (p3m_sr_forces_noalloc), called through the
C ABI, against the context-based path (p3m_sr_sort + p3m_sr_build_pairs +
p3m_sr_forces), on two calls in a row.

Callers that cannot allocate device memory (an application-owned memory pool,
a plugin handed only its input and output buffers) use this entry point; it
keeps its intermediate arrays in one fixed-size device array of the library.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from paper_2112_01508_gb300 import _native as nat
from tests._gpu_helpers import gpu_forces, rel_rms

pytestmark = pytest.mark.gpu

W = synth.workload("n32k")
FP32_TOL = 1e-5


def _params(w, n=None):
    p = nat.P3MParams()
    p.n = w.n if n is None else n
    p.box, p.x_s, p.x_r, p.G_m = 1.0, w.x_s, w.x_r, w.G_m
    p.softening, p.eps, p.n_rung = nat.SOFTENING["bspline"], w.eps, 8
    p.n_sub[0] = p.n_sub[1] = p.n_sub[2] = w.n_sub
    return p


def test_forces_noalloc_matches_context_path():
    pos = synth.workload_positions(W)
    ref = gpu_forces(pos, W.x_s, W.x_r, W.G_m, "bspline", W.eps, precision=32, n_sub=W.n_sub)["acc"]
    lib = nat.load()
    dev_pos = torch.from_numpy(pos.copy()).cuda()
    stream = torch.cuda.current_stream()
    params = _params(W)
    for call in range(2):
        out = torch.full((3, W.n), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.p3m_sr_forces_noalloc(ctypes.byref(params), ctypes.c_void_p(stream.cuda_stream),
                                       ctypes.c_void_p(dev_pos.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert st == nat.P3M_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all(), f"call {call}: non-finite output"
        assert rel_rms(got, ref) <= FP32_TOL, f"call {call}"
    # the input positions are not modified
    np.testing.assert_array_equal(dev_pos.cpu().numpy(), pos)


def test_forces_noalloc_rejects_oversized_input():
    lib = nat.load()
    params = _params(W, n=(1 << 16) + 1)
    out = torch.empty((3, 1), dtype=torch.float32, device="cuda")
    st = lib.p3m_sr_forces_noalloc(ctypes.byref(params), None, ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()))
    assert st == nat.P3M_ERR_INVALID
