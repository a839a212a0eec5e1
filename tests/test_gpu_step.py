"""GPU checks of the rung rule, kick, drift, permutation, VJP and error latch."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2112_01508_gb300 import ShortRange
from paper_2112_01508_gb300 import _native as nat
from tests._gpu_helpers import rel_rms

pytestmark = pytest.mark.gpu

W1 = synth.workload("n32k")


def _ctx(n, **kw):
    kw.setdefault("softening", "bspline")
    kw.setdefault("eps", W1.eps)
    return ShortRange(n, W1.x_s, W1.x_r, W1.G_m, **kw)


@pytest.mark.parametrize("prec", [32, 64])
def test_rungs_bitexact(prec):
    n = 100000
    mag = np.exp(synth.uniform(n, 1, 0, np.log(1e-4), np.log(1e6)))
    dirs = np.stack([synth.uniform(n, 1, (k + 1) * n, -1, 1) for k in range(3)])
    acc = (dirs * mag).astype(np.float32 if prec == 32 else np.float64)
    acc[:, :7] = [[0, 4.0 ** 0, 4.0 ** 3, np.nextafter(4.0 ** 3, 1e9), 1e30, 16.0, 0],
                  [0, 0, 0, 0, 0, 0, 0], [0, 0, 0, 0, 0, 0, 1e-30]]
    dt, eta, eps = 0.0123, 0.025, W1.eps
    with _ctx(n) as sr:
        got = sr.assign_rungs(torch.from_numpy(acc).cuda(), dt, eta, eps)
        sr.sync()
    ref, bad = oracle.rungs(acc.astype(np.float64), dt, eta, eps, 8)
    assert bad == 0
    np.testing.assert_array_equal(got.cpu().numpy(), ref)
    # boundary cases with dt^2 / (2 eta eps) = 1
    with _ctx(7) as sr:
        g2 = sr.assign_rungs(torch.from_numpy(np.ascontiguousarray(acc[:, :7])).cuda(), 1.0, 0.25, 2.0)
        sr.sync()
    r2, _ = oracle.rungs(acc[:, :7].astype(np.float64), 1.0, 0.25, 2.0, 8)
    np.testing.assert_array_equal(g2.cpu().numpy(), r2)


def test_nonfinite_acceleration_latched():
    acc = torch.zeros((3, 64), dtype=torch.float64, device="cuda")
    acc[0, 5] = float("nan")
    with _ctx(64) as sr:
        r = sr.assign_rungs(acc, 0.1, 0.025, 0.01)
        with pytest.raises(nat.P3MError) as e:
            sr.sync()
        assert e.value.status == nat.P3M_ERR_NONFINITE
        assert int(r[5]) == 0


def test_nonfinite_position_latched():
    pos = torch.rand((3, 256), dtype=torch.float64, device="cuda")
    pos[1, 3] = float("nan")
    pos[2, 9] = 1.5
    with _ctx(256) as sr:
        sr.sort(pos)
        with pytest.raises(nat.P3MError) as e:
            sr.sync()
        assert e.value.status == nat.P3M_ERR_NONFINITE


def test_call_order_enforced():
    with _ctx(16) as sr:
        pos = torch.rand((3, 16), dtype=torch.float64, device="cuda")
        with pytest.raises(nat.P3MError) as e:
            sr.forces(pos, 32)
        assert e.value.status == nat.P3M_ERR_STATE
        sr.sort(pos)
        with pytest.raises(nat.P3MError):
            sr.forces(pos, 32)  # build_pairs missing
        sr.build_pairs()
        sr.forces(pos, 32)
        sr.sync()


@pytest.mark.parametrize("mom_dt,acc_dt", [(np.float64, np.float32), (np.float64, np.float64),
                                           (np.float32, np.float32), (np.float32, np.float64)])
def test_kick_bitexact(mom_dt, acc_dt):
    n = 50000
    rng = np.random.default_rng(5)
    mom = rng.normal(size=(3, n)).astype(mom_dt)
    acc = rng.normal(size=(3, n)).astype(acc_dt)
    rung = synth.uniform_int8(n, 4, 0, 8)
    kf = [0.37 / 2 ** l for l in range(8)]
    with _ctx(n) as sr:
        m = torch.from_numpy(mom.copy()).cuda()
        sr.kick(m, torch.from_numpy(acc).cuda(), kf, torch.from_numpy(rung).cuda(), 2)
        sr.sync()
    ref = oracle.kick(mom.astype(np.float64), acc.astype(np.float64), kf, rung=rung, rung_min=2)
    np.testing.assert_array_equal(m.cpu().numpy(), ref.astype(mom_dt))


@pytest.mark.parametrize("mom_dt", [np.float64, np.float32])
def test_drift_bitexact(mom_dt):
    n = 50000
    rng = np.random.default_rng(6)
    pos = rng.random((3, n))
    mom = rng.normal(size=(3, n)).astype(mom_dt)
    with _ctx(n) as sr:
        p = torch.from_numpy(pos.copy()).cuda()
        sr.drift(p, torch.from_numpy(mom).cuda(), 0.0731)
        sr.sync()
    ref = oracle.drift(pos, mom.astype(np.float64), 0.0731)
    np.testing.assert_array_equal(p.cpu().numpy(), ref)


@pytest.mark.parametrize("mom_dt,acc_dt", [(np.float64, np.float32), (np.float64, np.float64),
                                           (np.float32, np.float32), (np.float32, np.float64)])
def test_kick_drift_bitexact(mom_dt, acc_dt):
    """The fused pass equals Eq. rung + kick + drift of the oracle, bit for bit, and
    the three separate entry points."""
    n = 60000
    rng = np.random.default_rng(9)
    pos = rng.random((3, n))
    pos[:, :50] = rng.choice([1e-17, 1.0 - 1e-16, 0.5], size=(3, 50))  # wraps at both faces
    mag = np.exp(rng.uniform(np.log(1e-3), np.log(1e6), n))
    acc = rng.normal(size=(3, n))
    acc = (acc * mag / np.linalg.norm(acc, axis=0)).astype(acc_dt)
    mom = rng.normal(size=(3, n)).astype(mom_dt)
    dt, eta, eps, drift = 0.0123, 0.025, W1.eps, 0.0731
    kf = [dt / 2 ** l for l in range(8)]
    rung_ref, bad = oracle.rungs(acc.astype(np.float64), dt, eta, eps, 8)
    assert bad == 0 and len(np.unique(rung_ref)) >= 5
    q_ref = oracle.kick(mom.astype(np.float64), acc.astype(np.float64), kf, rung=rung_ref, rung_min=0)
    q_ref = q_ref.astype(mom_dt)
    p_ref = oracle.drift(pos, q_ref.astype(np.float64), drift)
    with _ctx(n) as sr:
        p = torch.from_numpy(pos.copy()).cuda()
        m = torch.from_numpy(mom.copy()).cuda()
        a = torch.from_numpy(acc).cuda()
        r = torch.empty(n, dtype=torch.int8, device="cuda")
        sr.kick_drift(p, m, a, r, dt, eta, eps, kf, drift)
        # the same three steps as separate calls
        p2 = torch.from_numpy(pos.copy()).cuda()
        m2 = torch.from_numpy(mom.copy()).cuda()
        r2 = sr.assign_rungs(a, dt, eta, eps)
        sr.kick(m2, a, kf, r2, 0)
        sr.drift(p2, m2, drift)
        sr.sync()
    np.testing.assert_array_equal(r.cpu().numpy(), rung_ref)
    np.testing.assert_array_equal(m.cpu().numpy(), q_ref)
    np.testing.assert_array_equal(p.cpu().numpy(), p_ref)
    assert torch.equal(r, r2) and torch.equal(m, m2) and torch.equal(p, p2)


def test_kick_drift_keeps_the_sort_usable():
    """Forces after a fused kick-drift of the sorted positions (no new sort) equal the
    forces after a fresh sort: the pass records its displacement bound like a drift."""
    pos = synth.workload_positions(W1)
    n = W1.n
    with _ctx(n) as sr:
        p = torch.from_numpy(pos.copy()).cuda()
        sr.sort(p)
        sr.build_pairs()
        a = sr.forces(p, 64)
        m = torch.zeros((3, n), dtype=torch.float64, device="cuda")
        r = torch.empty(n, dtype=torch.int8, device="cuda")
        dt = 0.02
        sr.kick_drift(p, m, a, r, dt, 0.025, W1.eps, [dt / 2 ** l for l in range(8)], dt)
        sr.build_pairs()
        got = sr.forces(p, 64).cpu().numpy()
        pairs = sr.stats().pairs_last
        moved = p.cpu().numpy()
    ref, ref_pairs = oracle.sr_accel(moved, W1.x_s, W1.x_r, W1.G_m, "bspline", W1.eps)
    assert pairs == ref_pairs
    assert rel_rms(got, ref) <= 1e-12


def test_permute_roundtrip():
    pos = synth.workload_positions(W1)
    n = W1.n
    with _ctx(n) as sr:
        p = torch.from_numpy(pos.copy()).cuda()
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        sr.sort(p, perm_out=perm)
        x = torch.from_numpy(pos.copy()).cuda()
        xs = sr.permute(x)
        back = sr.unpermute(xs)
        sr.sync()
        np.testing.assert_array_equal(xs.cpu().numpy(), p.cpu().numpy())
        np.testing.assert_array_equal(back.cpu().numpy(), pos)


@pytest.mark.parametrize("softening", ["none", "plummer", "bspline"])
@pytest.mark.parametrize("rung_min", [None, 4])
def test_vjp_vs_oracle(softening, rung_min):
    pos = synth.workload_positions(W1)
    n = W1.n
    rung = synth.uniform_int8(n, 13, 0, 8) if rung_min is not None else None
    abar = np.stack([synth.uniform(n, 17, k * n, -1, 1) for k in range(3)])
    ref = oracle.sr_vjp(pos, abar, W1.x_s, W1.x_r, W1.G_m, softening, W1.eps, rung=rung,
                        rung_min=rung_min or 0)
    with _ctx(n, softening=softening) as sr:
        p = torch.from_numpy(pos.copy()).cuda()
        carry = []
        rg = None
        if rung is not None:
            rg = torch.from_numpy(rung.copy()).cuda()
            carry = [rg]
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        sr.sort(p, carry=carry, perm_out=perm)
        sr.build_pairs(rg, rung_min or 0)
        for prec, tol in ((64, 1e-12), (32, 1e-5)):
            dt = torch.float64 if prec == 64 else torch.float32
            ab = sr.permute(torch.from_numpy(abar).cuda().to(dt).contiguous())
            xb = sr.unpermute(sr.vjp(p, ab, prec))
            sr.sync()
            err = rel_rms(xb.cpu().numpy(), ref)
            if softening == "none" and prec == 32:
                assert err < 1e-3
            else:
                assert err <= tol, (prec, err)


@pytest.mark.parametrize("rung_min", [None, 4])
def test_vjp_each_pair_once_matches_one_sided(rung_min):
    """FP32 adjoint: the each-pair-once kernel (the pair term J_ij (v_i - v_j) is
    antisymmetric, so the partner gets the negated term) and the one-sided kernel
    both match the oracle, agree with each other, and their gradients sum to zero."""
    pos = synth.workload_positions(W1)
    n = W1.n
    rung = synth.uniform_int8(n, 13, 0, 8) if rung_min is not None else None
    abar = np.stack([synth.uniform(n, 19, k * n, -1, 1) for k in range(3)])
    ref = oracle.sr_vjp(pos, abar, W1.x_s, W1.x_r, W1.G_m, "bspline", W1.eps, rung=rung,
                        rung_min=rung_min or 0)
    got = {}
    for sym in (True, False):
        with _ctx(n, symmetric=sym) as sr:
            p = torch.from_numpy(pos.copy()).cuda()
            rg = None
            carry = []
            if rung is not None:
                rg = torch.from_numpy(rung.copy()).cuda()
                carry = [rg]
            sr.sort(p, carry=carry)
            sr.build_pairs(rg, rung_min or 0)
            ab = sr.permute(torch.from_numpy(abar).cuda().float().contiguous())
            xb = sr.unpermute(sr.vjp(p, ab, 32))
            sr.sync()
            got[sym] = xb.double().cpu().numpy()
        assert np.isfinite(got[sym]).all()
        assert rel_rms(got[sym], ref) <= 1e-5, (sym, rel_rms(got[sym], ref))
        assert np.abs(got[sym].sum(axis=1)).max() <= 1e-6 * np.abs(got[sym]).sum(axis=1).max()
    # two FP32 sums in different orders, each ~1e-6 from the FP64 oracle on this set
    # (the adjoint's v_i - v_j and D terms cancel more than the force's terms)
    assert rel_rms(got[True], got[False]) <= 5e-6


@pytest.mark.parametrize("softening", ["plummer", "bspline"])
def test_vjp_dense_cluster_with_coincident_particles(softening):
    """FP32 adjoint on a dense cluster in which most pairs are closer than r_sw (most
    steps take the packed softened branch with its derivative) and 40 particles sit
    exactly on others (r = 0: the softened B(0) acts on abar_i - abar_j), against the
    oracle: the each-pair-once and the one-sided kernels, with every particle active
    and on a partial set (abar masked to the receivers)."""
    rng = np.random.default_rng(23)
    x_r, eps = 0.1, 0.004
    dense = 0.4 + 2e-3 * rng.normal(size=(3, 1500))
    pos = np.concatenate([dense, rng.random((3, 1000)), dense[:, :40]], axis=1) % 1.0
    n = pos.shape[1]
    abar = rng.normal(size=(3, n))
    rung = synth.uniform_int8(n, 29, 0, 8)
    for symmetric, rung_min in ((True, None), (False, None), (True, 5), (False, 5)):
        ref = oracle.sr_vjp(pos, abar, x_r / 4.5, x_r, 1.0 / n, softening, eps,
                            rung=rung if rung_min else None, rung_min=rung_min or 0)
        with ShortRange(n, x_r / 4.5, x_r, 1.0 / n, softening=softening, eps=eps, symmetric=symmetric) as sr:
            p = torch.from_numpy(pos.copy()).cuda()
            rg = torch.from_numpy(rung.copy()).cuda() if rung_min else None
            sr.sort(p, carry=[rg] if rg is not None else [])
            sr.build_pairs(rg, rung_min or 0)
            ab = sr.permute(torch.from_numpy(abar).cuda().float().contiguous())
            xb = sr.unpermute(sr.vjp(p, ab, 32)).double().cpu().numpy()
        assert np.isfinite(xb).all()
        assert rel_rms(xb, ref) <= 1e-5, (symmetric, rung_min, rel_rms(xb, ref))
