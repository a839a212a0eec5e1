"""GPU rung-based leapfrog (Section 2.2.2) against the oracle's cycle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2112_01508_gb300 import ShortRange
from paper_2112_01508_gb300.integrate import rung_leapfrog, substep_rung_min
from tests._gpu_helpers import rel_rms

pytestmark = pytest.mark.gpu

W = synth.workload("n32k")


def _subset(n, seed):
    full = synth.workload_positions(W)
    idx = np.random.default_rng(seed).choice(W.n, size=n, replace=False)
    return np.ascontiguousarray(full[:, idx])


def _dt_for_rungs(pos, eta, eps):
    """A step for which the median particle sits on rung 1 of Eq. rung."""
    acc, _ = oracle.sr_accel(pos, W.x_s, W.x_r, W.G_m, "bspline", eps)
    a = np.sqrt((acc ** 2).sum(axis=0))
    return 2.0 * float(np.sqrt(2 * eta * eps / np.median(a)))


@pytest.mark.parametrize("n_rung,n_steps,period,resort", [(4, 2, None, 1), (3, 3, None, 1), (4, 4, 2, 1),
                                                         (4, 2, None, 4), (3, 3, 2, 3)])
def test_rung_leapfrog_vs_oracle(n_rung, n_steps, period, resort):
    n, eta, eps = 4096, 0.025, W.eps
    pos = _subset(n, 5)
    dt = _dt_for_rungs(pos, eta, eps)
    p_ref, q_ref, rung_ref, state_ref, hist_ref = oracle.rung_leapfrog(
        pos, np.zeros_like(pos), W.x_s, W.x_r, W.G_m, "bspline", eps, dt, eta, n_rung, n_steps, period=period)
    # the run must exercise several rungs and jumps
    assert len(np.unique(hist_ref[0])) >= 3
    assert sum(int((a != b).sum()) for a, b in zip(hist_ref[:-1], hist_ref[1:])) > 0
    dev = torch.device("cuda")
    with ShortRange(n, W.x_s, W.x_r, W.G_m, softening="bspline", eps=eps, n_sub=W.n_sub, n_rung=n_rung) as sr:
        p = torch.from_numpy(pos.copy()).to(dev)
        q = torch.zeros_like(p)
        ids = torch.arange(n, dtype=torch.int32, device=dev)
        hist = []
        rung, state = rung_leapfrog(sr, p, q, dt, eta, eps, n_steps, precision=64, period=period, carry=(ids,),
                                    history=hist, resort_every=resort)
        sr.sync()
        order = ids.cpu().numpy().astype(np.int64)
        got_p = np.empty_like(pos)
        got_q = np.empty_like(pos)
        got_p[:, order] = p.cpu().numpy()
        got_q[:, order] = q.cpu().numpy()
        got_rung = np.empty(n, np.int8)
        got_rung[order] = rung.cpu().numpy()
        got_state = np.empty(n, np.int8)
        got_state[order] = state.cpu().numpy()
    np.testing.assert_array_equal(got_rung, rung_ref)
    np.testing.assert_array_equal(got_state, state_ref)
    assert np.all(got_state == 0)
    # FP64 forces agree with the oracle to ~1e-13 relative; two to three steps keep that far below 1e-10
    dp = got_p - p_ref
    dp -= np.round(dp)  # periodic wrap
    assert np.abs(dp).max() <= 1e-10 * W.x_r
    assert np.abs(got_q - q_ref).max() <= 1e-10 * np.abs(q_ref).max()


def test_substep_rung_min():
    assert [substep_rung_min(k, 4) for k in range(1, 9)] == [3, 2, 3, 1, 3, 2, 3, 0]
    assert [substep_rung_min(k, 1) for k in range(1, 4)] == [0, 0, 0]


def test_rung_kick_rejects_bad_rung_and_order():
    n = 256
    dev = torch.device("cuda")
    with ShortRange(n, W.x_s, W.x_r, W.G_m, softening="bspline", eps=W.eps, n_rung=4) as sr:
        mom = torch.zeros((3, n), dtype=torch.float64, device=dev)
        acc = torch.ones((3, n), dtype=torch.float64, device=dev)
        rung = torch.zeros(n, dtype=torch.int8, device=dev)
        state = torch.zeros(n, dtype=torch.int8, device=dev)
        from paper_2112_01508_gb300 import _native as nat
        # rung_min must match the substep counter
        with pytest.raises(nat.P3MError) as e:
            sr.rung_kick(mom, acc, rung, state, 2, 8, 0.1, 0.025, W.eps)
        assert e.value.status == nat.P3M_ERR_INVALID
        # synchronisation only at the end of a global step
        with pytest.raises(nat.P3MError):
            sr.rung_kick(mom, acc, rung, state, 3, 3, 0.1, 0.025, W.eps, synchronize=True)
        rung[7] = 9
        sr.rung_kick(mom, acc, rung, state, 0, 8, 0.1, 0.025, W.eps)
        with pytest.raises(nat.P3MError) as e:
            sr.sync()
        assert e.value.status == nat.P3M_ERR_STATE
        assert float(mom[:, 7].abs().max()) == 0.0
        assert float(mom[:, 6].abs().min()) > 0.0


def test_rung_leapfrog_with_long_range_vs_oracle():
    """The full P3M cycle: short-range rung kicks plus the mesh force on every rung-0 kick."""
    from paper_2112_01508_gb300 import LongRange
    n, eta, eps, n_rung, n_steps, n_phi = 4096, 0.025, W.eps, 3, 2, 32
    pos = _subset(n, 7)
    dt = _dt_for_rungs(pos, eta, eps)
    p_ref, q_ref, rung_ref, _, _ = oracle.rung_leapfrog(
        pos, np.zeros_like(pos), W.x_s, W.x_r, W.G_m, "bspline", eps, dt, eta, n_rung, n_steps, n_phi=n_phi)
    dev = torch.device("cuda")
    with ShortRange(n, W.x_s, W.x_r, W.G_m, softening="bspline", eps=eps, n_sub=W.n_sub, n_rung=n_rung) as sr, \
            LongRange(n, n_phi, W.x_s, W.G_m, precision=64) as lr:
        p = torch.from_numpy(pos.copy()).to(dev)
        q = torch.zeros_like(p)
        ids = torch.arange(n, dtype=torch.int32, device=dev)
        rung, _ = rung_leapfrog(sr, p, q, dt, eta, eps, n_steps, precision=64, carry=(ids,), long_range=lr)
        sr.sync()
        lr.sync()
        order = ids.cpu().numpy().astype(np.int64)
        got_p = np.empty_like(pos)
        got_q = np.empty_like(pos)
        got_p[:, order] = p.cpu().numpy()
        got_q[:, order] = q.cpu().numpy()
        got_rung = np.empty(n, np.int8)
        got_rung[order] = rung.cpu().numpy()
    np.testing.assert_array_equal(got_rung, rung_ref)
    dp = got_p - p_ref
    dp -= np.round(dp)
    assert np.abs(dp).max() <= 1e-10 * W.x_r
    assert np.abs(got_q - q_ref).max() <= 1e-10 * np.abs(q_ref).max()


@pytest.mark.parametrize("mom_dt,acc_dt", [(np.float64, np.float64), (np.float64, np.float32),
                                           (np.float32, np.float32), (np.float32, np.float64)])
@pytest.mark.parametrize("k,sync", [(1, False), (2, False), (4, False), (6, False), (8, True)])
def test_rung_kick_bitexact(mom_dt, acc_dt, k, sync):
    """One rung kick against the oracle's: momenta (rounded once to FP32 where stored
    in FP32), rungs and kick states bit for bit, jumps in both directions included."""
    n, n_rung, dt, eta, eps = 50000, 4, 0.07, 0.025, W.eps
    rng = np.random.default_rng(k)
    mag = np.exp(rng.uniform(np.log(1e-3), np.log(1e5), n))
    acc = rng.normal(size=(3, n))
    acc = (acc * mag / np.linalg.norm(acc, axis=0)).astype(acc_dt)
    mom = rng.normal(size=(3, n)).astype(mom_dt)
    rung = rng.integers(0, n_rung, n).astype(np.int8)
    state = rng.integers(0, 3, n).astype(np.int8)
    tz = 0
    while tz < n_rung - 1 and (k >> tz) & 1 == 0:
        tz += 1
    lmin = n_rung - 1 - tz
    q_ref = mom.astype(np.float64).copy()
    r_ref, s_ref = rung.copy(), state.copy()
    oracle.rung_kick(q_ref, acc.astype(np.float64), r_ref, s_ref, lmin, k, n_rung, dt, eta, eps, sync)
    with ShortRange(n, W.x_s, W.x_r, W.G_m, softening="bspline", eps=eps, n_rung=n_rung) as sr:
        q = torch.from_numpy(mom.copy()).cuda()
        r = torch.from_numpy(rung.copy()).cuda()
        s = torch.from_numpy(state.copy()).cuda()
        sr.rung_kick(q, torch.from_numpy(acc).cuda(), r, s, lmin, k, dt, eta, eps, synchronize=sync)
        sr.sync()
        got_q, got_r, got_s = q.cpu().numpy(), r.cpu().numpy(), s.cpu().numpy()
    np.testing.assert_array_equal(got_q, q_ref.astype(mom_dt))
    np.testing.assert_array_equal(got_r, r_ref)
    np.testing.assert_array_equal(got_s, s_ref)
    if not sync:
        assert (got_r != rung).any()  # some particles jumped


# FP32 rung cycle against the FP64 oracle cycle (the bounds below are derived in the
# design notes, reading "FP32 rung cycle"):
FP32_CYCLE_MAX_RUNG_CHANGES = 4   # particles whose rung history may differ (0.1% of 4096)
FP32_CYCLE_DX = 1e-4              # per-particle |dx| / largest displacement of the oracle cycle
FP32_CYCLE_DQ = 2e-4              # per-particle |dq| / largest momentum of the oracle cycle
FP32_CYCLE_RMS = 1e-5             # relative RMS of displacements and momenta


def test_rung_leapfrog_fp32_momenta_vs_oracle():
    """FP32 momenta (stored once rounded after each FP64 kick) and FP32 forces: the
    cycle stays within FP32 rounding, grown by the dynamics, of the FP64 oracle cycle.

    A particle whose FP32 acceleration lies within FP32 rounding of a power-of-16
    boundary of Eq. rung may take the other rung (and kick schedule); there may be at
    most FP32_CYCLE_MAX_RUNG_CHANGES such particles, and they and their neighbours
    (which met them on another trajectory) are left out of the per-particle bounds."""
    n, eta, eps, n_rung, n_steps = 4096, 0.025, W.eps, 4, 2
    pos = _subset(n, 11)
    dt = _dt_for_rungs(pos, eta, eps)
    p_ref, q_ref, _, _, hist_ref = oracle.rung_leapfrog(
        pos, np.zeros_like(pos), W.x_s, W.x_r, W.G_m, "bspline", eps, dt, eta, n_rung, n_steps)
    dev = torch.device("cuda")
    with ShortRange(n, W.x_s, W.x_r, W.G_m, softening="bspline", eps=eps, n_sub=W.n_sub, n_rung=n_rung) as sr:
        p = torch.from_numpy(pos.copy()).to(dev)
        q = torch.zeros((3, n), dtype=torch.float32, device=dev)
        ids = torch.arange(n, dtype=torch.int32, device=dev)
        hist, orders = [], []
        rung_leapfrog(sr, p, q, dt, eta, eps, n_steps, precision=32, carry=(ids,), resort_every=2, history=hist,
                      on_substep=lambda k, lmin: orders.append(ids.clone()))
        sr.sync()
        order = ids.cpu().numpy().astype(np.int64)
        got_p = np.empty_like(pos)
        got_q = np.empty_like(pos)
        got_p[:, order] = p.cpu().numpy()
        got_q[:, order] = q.double().cpu().numpy()
    # per-particle rung histories in the caller's order
    same = np.ones(n, bool)
    assert len(hist) == len(hist_ref) == len(orders)
    for h_gpu, o_gpu, h_ref in zip(hist, orders, hist_ref):
        h = np.empty(n, np.int8)
        h[o_gpu.cpu().numpy().astype(np.int64)] = h_gpu.cpu().numpy()
        same &= h == h_ref
    changed = np.flatnonzero(~same)
    assert len(changed) <= FP32_CYCLE_MAX_RUNG_CHANGES, len(changed)
    d_got = got_p - pos
    d_got -= np.round(d_got)
    d_ref = p_ref - pos
    d_ref -= np.round(d_ref)
    X = np.linalg.norm(d_ref, axis=0).max()
    Q = np.linalg.norm(q_ref, axis=0).max()
    # neighbours of a particle on another rung history: within x_r + 2X of it at the start
    clean = same.copy()
    for c in changed:
        dd = pos - pos[:, c:c + 1]
        dd -= np.round(dd)
        clean &= np.sqrt((dd ** 2).sum(axis=0)) >= W.x_r + 2 * X
    assert clean.sum() >= n - 129 * len(changed)
    dx = np.linalg.norm(d_got - d_ref, axis=0)
    dq = np.linalg.norm(got_q - q_ref, axis=0)
    assert dx[clean].max() <= FP32_CYCLE_DX * X, dx[clean].max() / X
    assert dq[clean].max() <= FP32_CYCLE_DQ * Q, dq[clean].max() / Q
    assert rel_rms(d_got[:, clean], d_ref[:, clean]) <= FP32_CYCLE_RMS
    assert rel_rms(got_q[:, clean], q_ref[:, clean]) <= FP32_CYCLE_RMS


@pytest.mark.parametrize("mom_dt,acc_dt", [(np.float64, np.float32), (np.float32, np.float64)])
@pytest.mark.parametrize("k", [1, 2, 4])
def test_rung_kick_drift_equals_kick_then_drift(mom_dt, acc_dt, k):
    """The fused kick + drift pass gives the momenta, rungs, kick states and positions of
    p3m_sr_rung_kick followed by p3m_sr_drift, bit for bit."""
    n, n_rung, dt, eta, eps = 50000, 4, 0.07, 0.025, W.eps
    rng = np.random.default_rng(40 + k)
    mag = np.exp(rng.uniform(np.log(1e-3), np.log(1e5), n))
    acc = rng.normal(size=(3, n))
    acc = (acc * mag / np.linalg.norm(acc, axis=0)).astype(acc_dt)
    mom = rng.normal(size=(3, n)).astype(mom_dt)
    pos = rng.random((3, n))
    pos[:, :20] = 1.0 - 1e-16  # wraps
    rung = rng.integers(0, n_rung, n).astype(np.int8)
    state = rng.integers(0, 3, n).astype(np.int8)
    tz = 0
    while tz < n_rung - 1 and (k >> tz) & 1 == 0:
        tz += 1
    lmin = n_rung - 1 - tz
    with ShortRange(n, W.x_s, W.x_r, W.G_m, softening="bspline", eps=eps, n_rung=n_rung) as sr:
        t = lambda a: torch.from_numpy(a.copy()).cuda()
        q1, r1, s1, p1 = t(mom), t(rung), t(state), t(pos)
        sr.rung_kick_drift(q1, t(acc), r1, s1, lmin, k, dt, eta, eps, p1, dt / 8)
        q2, r2, s2, p2 = t(mom), t(rung), t(state), t(pos)
        sr.rung_kick(q2, t(acc), r2, s2, lmin, k, dt, eta, eps)
        sr.drift(p2, q2, dt / 8)
        sr.sync()
    for a, b in ((q1, q2), (r1, r2), (s1, s2), (p1, p2)):
        assert torch.equal(a, b)
    assert (r1.cpu().numpy() != rung).any()
