"""The allocation-free entry point (p3m_sr_forces_noalloc), called through the
C ABI, against the CPU oracle and against the context-based path
(p3m_sr_sort + p3m_sr_build_pairs + p3m_sr_forces).

Callers that cannot allocate device memory (an application-owned memory pool,
a plugin handed only its input and output buffers, a pipeline that forbids
cudaMalloc after start-up) use this entry point; it keeps its intermediate
arrays in one fixed-size device array of the library, shared by every call, so
each case below makes two calls in a row and checks both.  Its size limits are
checked without a GPU in test_abi_cpu.py (the rejections happen before any
device call).  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2112_01508_gb300 import _native as nat
from tests._gpu_helpers import gpu_forces, rel_rms

pytestmark = pytest.mark.gpu

W = synth.workload("n32k")
FP32_TOL = 1e-5     # relative RMS force of the FP32 path against the FP64 oracle
MAX_N = 1 << 16     # the entry point's particle limit


def _params(n, n_sub=None):
    p = nat.P3MParams()
    p.n = n
    p.box, p.x_s, p.x_r, p.G_m = 1.0, W.x_s, W.x_r, W.G_m
    p.softening, p.eps, p.n_rung = nat.SOFTENING["bspline"], W.eps, 8
    p.n_sub[0] = p.n_sub[1] = p.n_sub[2] = W.n_sub if n_sub is None else n_sub
    return p


def _noalloc(pos_dev, n, calls=2):
    """Run the entry point `calls` times on the same input; return each output."""
    lib = nat.load()
    stream = torch.cuda.current_stream()
    params = _params(n)
    outs = []
    for _ in range(calls):
        out = torch.full((3, max(n, 1)), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.p3m_sr_forces_noalloc(ctypes.byref(params), ctypes.c_void_p(stream.cuda_stream),
                                       ctypes.c_void_p(pos_dev.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert st == nat.P3M_OK
        torch.cuda.synchronize()
        outs.append(out[:, :n].cpu().numpy().astype(np.float64))
    return outs


def _check_against_oracle(pos, outs, ref):
    for call, got in enumerate(outs):
        assert np.isfinite(got).all(), f"call {call}: non-finite output"
        assert rel_rms(got, ref) <= FP32_TOL, f"call {call}: rel RMS {rel_rms(got, ref)}"


def test_forces_noalloc_vs_oracle_and_context_path():
    pos = synth.workload_positions(W)
    ref, _ = oracle.sr_accel(pos, W.x_s, W.x_r, W.G_m, "bspline", W.eps)
    dev_pos = torch.from_numpy(pos.copy()).cuda()
    outs = _noalloc(dev_pos, W.n)
    _check_against_oracle(pos, outs, ref)
    # second check: the context path (sort, work list, FP32 forces) on the same input
    ctx = gpu_forces(pos, W.x_s, W.x_r, W.G_m, "bspline", W.eps, precision=32, n_sub=W.n_sub)["acc"]
    for got in outs:
        assert rel_rms(got, ctx) <= FP32_TOL
    # the input positions are not modified
    np.testing.assert_array_equal(dev_pos.cpu().numpy(), pos)


def test_forces_noalloc_at_the_particle_limit():
    """n = 2^16, the largest set the internal array holds (clustered as the 32^3 recipe)."""
    pos = synth.positions(MAX_N, 2024, W.frac_uniform, W.n_spheres, W.b_lo, W.b_hi)
    ref, _ = oracle.sr_accel(pos, W.x_s, W.x_r, W.G_m, "bspline", W.eps)
    outs = _noalloc(torch.from_numpy(pos.copy()).cuda(), MAX_N)
    _check_against_oracle(pos, outs, ref)


@pytest.mark.parametrize("n", [1, 2, 33])
def test_forces_noalloc_small_ragged_sets(n):
    """One particle, one pair, and one full chunk of 32 receivers plus a ragged one,
    all inside one small Plummer sphere so that (nearly) every pair interacts."""
    pos = synth.positions(n, 77 + n, 0.0, 1, 0.002, 0.002)
    ref, pairs = oracle.sr_accel(pos, W.x_s, W.x_r, W.G_m, "bspline", W.eps)
    outs = _noalloc(torch.from_numpy(pos.copy()).cuda(), n)
    if n == 1:
        for got in outs:
            np.testing.assert_array_equal(got, np.zeros((3, 1)))
        return
    assert pairs >= 0.9 * n * (n - 1)
    _check_against_oracle(pos, outs, ref)


def test_forces_noalloc_empty_set():
    lib = nat.load()
    params = _params(0)
    st = lib.p3m_sr_forces_noalloc(ctypes.byref(params), None, None, None)
    assert st == nat.P3M_OK


def test_forces_noalloc_periodic_images_and_nonfinite_particles():
    """The box is periodic: positions shifted by whole box lengths give the forces of
    their images.  A particle with a non-finite coordinate gets NaN accelerations and
    exerts no force on the others."""
    n = 4096
    pos = synth.positions(n, 31, W.frac_uniform, W.n_spheres, W.b_lo, W.b_hi)
    shifted = pos.copy()
    rng = np.random.default_rng(5)
    moved = rng.choice(n, size=300, replace=False)
    shifted[:, moved] += rng.integers(-3, 4, size=(3, 300)).astype(np.float64)
    bad = np.array([17, 2500])
    shifted[0, bad[0]] = np.nan
    shifted[2, bad[1]] = np.inf
    keep = np.setdiff1d(np.arange(n), bad)
    ref_keep, _ = oracle.sr_accel(np.ascontiguousarray(pos[:, keep]), W.x_s, W.x_r, W.G_m, "bspline", W.eps)
    outs = _noalloc(torch.from_numpy(shifted).cuda(), n)
    for got in outs:
        assert np.isnan(got[:, bad]).all()
        assert np.isfinite(got[:, keep]).all()
        assert rel_rms(got[:, keep], ref_keep) <= FP32_TOL
