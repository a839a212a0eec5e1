"""GPU parity of the long-range mesh library (include/p3m_pm.h) against the PM
oracle (oracle/pm.py), step by step and end to end."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import pm as opm
from paper_2112_01508_gb300 import LongRange, ShortRange
from paper_2112_01508_gb300 import _native as nat
from tests._gpu_helpers import rel_rms

pytestmark = pytest.mark.gpu

W = synth.workload("n32k")
FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def n32k():
    return synth.workload_positions(W)


def _lr(pos, n_phi, x_s, G_m, p_i=2, p_d=4, precision=64, **kw):
    with LongRange(pos.shape[1], n_phi, x_s, G_m, p_i=p_i, p_d=p_d, precision=precision) as lr:
        p = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
        a = lr.accel(p)
        phi = lr.potential()
        rho = lr.assign(p)
        lr.sync()
        return a.double().cpu().numpy(), phi.double().cpu().numpy(), rho.double().cpu().numpy()


@pytest.mark.parametrize("precision,tol", [(64, FP64_TOL), (32, FP32_TOL)])
def test_mesh_steps_and_accel_match_oracle(n32k, precision, tol):
    pos = n32k
    n_phi, x_s, G_m = W.n_phi, W.x_s, W.G_m
    a, phi, rho = _lr(pos, n_phi, x_s, G_m, precision=precision)
    rho_ref = opm.assign(pos, n_phi, 2)
    assert rel_rms(rho, rho_ref) <= (1e-14 if precision == 64 else 1e-6)
    phi_ref = 4 * np.pi * G_m * n_phi ** 4 * opm.potential_mesh(rho_ref, x_s, 2)
    assert rel_rms(phi, phi_ref) <= tol
    ref = opm.lr_accel(pos, n_phi, x_s, G_m)
    err = rel_rms(a, ref)
    print(f"precision {precision}: accel rel RMS {err:.3e}")
    assert err <= tol


@pytest.mark.parametrize("p_i,p_d", [(1, 2), (2, 2), (3, 6), (4, 8), (4, 4), (3, 2)])
def test_orders_match_oracle(n32k, p_i, p_d):
    pos = np.ascontiguousarray(n32k[:, :4096])
    n_phi = 32
    x_s = 1.25 / n_phi
    a, _, rho = _lr(pos, n_phi, x_s, 1.0 / 4096, p_i=p_i, p_d=p_d)
    assert rel_rms(rho, opm.assign(pos, n_phi, p_i)) <= 1e-14
    assert rel_rms(a, opm.lr_accel(pos, n_phi, x_s, 1.0 / 4096, p_i=p_i, p_d=p_d)) <= FP64_TOL


def test_plain_pm_poisson_kernel(n32k):
    pos = np.ascontiguousarray(n32k[:, :2048])
    a, _, _ = _lr(pos, 32, 0.0, 1.0 / 2048, p_i=2, p_d=2)
    assert rel_rms(a, opm.lr_accel(pos, 32, 0.0, 1.0 / 2048, p_i=2, p_d=2)) <= FP64_TOL


def test_momentum_conservation_and_accumulate(n32k):
    pos = n32k
    with LongRange(W.n, W.n_phi, W.x_s, W.G_m, precision=64) as lr:
        p = torch.from_numpy(pos.copy()).cuda()
        a = lr.accel(p)
        assert float(a.sum(dim=1).abs().max()) <= 1e-12 * float(a.abs().sum())
        base = torch.randn((3, W.n), dtype=torch.float64, device="cuda")
        out = base.clone()
        lr.accel(p, out, accumulate=True)
        lr.sync()
        # the second call's atomics may sum the mesh in another order: compare to rounding
        torch.testing.assert_close(out, base + a, rtol=1e-14, atol=1e-12 * float(a.abs().max()))


def test_ragged_and_empty_sets():
    rng = np.random.default_rng(4)
    for n in (0, 1, 7, 1001):
        pos = rng.random((3, n))
        with LongRange(n, 16, 1.25 / 16, 1.0, precision=64) as lr:
            p = torch.from_numpy(pos).cuda()
            a = lr.accel(p)
            lr.sync()
            if n:
                ref = opm.lr_accel(pos, 16, 1.25 / 16, 1.0)
                # scale: G m n / L_phi^2 (one particle's self-force is zero up to rounding)
                np.testing.assert_allclose(a.cpu().numpy(), ref, rtol=0, atol=1e-12 * n * 16.0 ** 2)


def test_bad_positions_latch_and_contribute_nothing(n32k):
    pos = np.ascontiguousarray(n32k[:, :4096]).copy()
    bad = [5, 77, 300]
    pos[0, 5] = np.nan
    pos[1, 77] = 1.0          # outside [0, L)
    pos[2, 300] = -1e-9
    good = np.setdiff1d(np.arange(4096), bad)
    with LongRange(4096, 32, 1.25 / 32, 1.0 / 4096, precision=64) as lr:
        p = torch.from_numpy(pos).cuda()
        a = lr.accel(p)
        with pytest.raises(nat.P3MError) as e:
            lr.sync()
        assert e.value.status == nat.P3M_ERR_NONFINITE
        a = a.cpu().numpy()
        lr.sync()  # the latch is cleared once reported
    assert np.all(a[:, bad] == 0)
    ref = opm.lr_accel(pos[:, good], 32, 1.25 / 32, 1.0 / 4096)
    assert rel_rms(a[:, good], ref) <= FP64_TOL


def test_potential_before_accel_is_a_state_error():
    with LongRange(10, 16, 0.1, 1.0) as lr:
        with pytest.raises(nat.P3MError) as e:
            lr.potential()
        assert e.value.status == nat.P3M_ERR_STATE


def test_p3m_total_force_matches_ewald():
    """Short-range (GPU, FP64) plus long-range (GPU, FP64) against the exact periodic
    force of an Ewald sum: the P3M split at the paper's parameters (x_s = 1.25 L_phi,
    x_r = 4.5 x_s, CIC, D_4) is accurate to well under a percent of the total force."""
    rng = np.random.default_rng(8)
    n = 128
    pos = rng.random((3, n))
    n_phi = 32
    x_s = 1.25 / n_phi
    x_r = 4.5 * x_s
    G_m = 1.0 / n
    p = torch.from_numpy(pos.copy()).cuda()
    with LongRange(n, n_phi, x_s, G_m, precision=64) as lr:
        a_lr = lr.accel(p).cpu().numpy()
    with ShortRange(n, x_s, x_r, G_m, softening="none", n_sub=1) as sr:
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        ps = p.clone()
        sr.sort(ps, perm_out=perm)
        sr.build_pairs()
        a = sr.forces(ps, 64)
        a_sr = np.empty((3, n))
        a_sr[:, perm.cpu().numpy().astype(np.int64)] = a.cpu().numpy()
    # exact: short-range without truncation (cut where erfc < 1e-16) + reciprocal sum
    xs2 = 0.02
    exact = oracle.sr_accel(pos, xs2, 0.25, G_m, "none", 0.0)[0] + opm.ewald_lr_exact(pos, xs2, G_m)
    err = rel_rms(a_sr + a_lr, exact)
    print("P3M total force rel RMS vs Ewald:", err)
    assert err <= 5e-3
