"""Differentiable path: autograd Function over the adjoint kernel and the
checkpointed 16-step leapfrog, against finite differences and the oracle's
analytic gradient."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2112_01508_gb300 import ShortRange
from paper_2112_01508_gb300.autograd import leapfrog, short_range_accel

pytestmark = pytest.mark.gpu


def _setup(w, n_take=None, seed=3):
    pos = synth.workload_positions(w)
    if n_take:
        idx = np.random.default_rng(seed).choice(w.n, size=n_take, replace=False)
        pos = np.ascontiguousarray(pos[:, idx])
    return pos


def _dt(acc, eps, eta=0.025):
    """Uniform time step from the rung criterion (Eq. rung): rung 0 for 99% of the
    particles, dt = sqrt(2 eta eps / Q_0.99(|a|))."""
    amag = np.sqrt((acc ** 2).sum(axis=0))
    return float(np.sqrt(2 * eta * eps / np.quantile(amag, 0.99)))


def test_accel_gradcheck_against_vjp_oracle():
    w = synth.workload("n32k")
    pos = _setup(w)
    n = pos.shape[1]
    abar = np.stack([synth.uniform(n, 3, k * n, -1, 1) for k in range(3)])
    with ShortRange.from_workload(w) as sr:
        x = torch.from_numpy(pos.copy()).cuda().requires_grad_(True)
        a = short_range_accel(x, sr, 64)
        (a * torch.from_numpy(abar).cuda()).sum().backward()
        got = x.grad.cpu().numpy()
    ref = oracle.sr_vjp(pos, abar, w.x_s, w.x_r, w.G_m, "bspline", w.eps)
    err = np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum())
    assert err <= 1e-12


def _oracle_leapfrog_grad(pos, w, dt, n_steps, wts):
    """d(sum w . x_N)/d x_0 through the KDK leapfrog, by the oracle's forward and VJP."""
    def acc(x):
        return oracle.sr_accel(x, w.x_s, w.x_r, w.G_m, "bspline", w.eps)[0]

    xs, qs = [pos.copy()], []
    q = np.zeros_like(pos)
    a = acc(pos)
    x = pos.copy()
    traj = []
    for _ in range(n_steps):
        q = q + 0.5 * dt * a
        xn = x + dt * q
        xn = xn - np.floor(xn)
        traj.append((x, q.copy()))
        x = xn
        a = acc(x)
        q = q + 0.5 * dt * a
        xs.append(x.copy())
    # reverse pass: state (xbar, qbar), a_k = acc(x_k)
    xbar = wts.copy()
    qbar = np.zeros_like(pos)
    for s in range(n_steps - 1, -1, -1):
        x_new = xs[s + 1]
        # q_{s+1} = q_half + dt/2 a(x_new)
        abar = 0.5 * dt * qbar
        xbar = xbar + oracle.sr_vjp(x_new, abar, w.x_s, w.x_r, w.G_m, "bspline", w.eps)
        # x_new = x_s + dt q_half
        qbar = qbar + dt * xbar
        # q_half = q_s + dt/2 a(x_s)
        abar = 0.5 * dt * qbar
        xbar = xbar + oracle.sr_vjp(xs[s], abar, w.x_s, w.x_r, w.G_m, "bspline", w.eps)
    return xbar


def test_leapfrog_gradient_vs_oracle_analytic():
    w = synth.workload("n32k")
    pos = _setup(w)
    acc0 = oracle.sr_accel(pos, w.x_s, w.x_r, w.G_m, "bspline", w.eps)[0]
    dt = _dt(acc0, w.eps)
    n = pos.shape[1]
    wts = np.stack([synth.uniform(n, 8, k * n, -1, 1) for k in range(3)])
    ref = _oracle_leapfrog_grad(pos, w, dt, 16, wts)
    with ShortRange.from_workload(w) as sr:
        x0 = torch.from_numpy(pos.copy()).cuda().requires_grad_(True)
        q0 = torch.zeros_like(x0)
        x16, _ = leapfrog(x0, q0, sr, dt, 16, 4, precision=64)
        (x16 * torch.from_numpy(wts).cuda()).sum().backward()
        got = x0.grad.cpu().numpy()
    err = np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum())
    assert err <= 1e-9, err


def _trajectory(x, sr, dt, n_steps, states=None):
    """The leapfrog's KDK sequence without autograd, recording the interacting
    pair count of every force evaluation (and optionally the positions)."""
    from paper_2112_01508_gb300.autograd import Drift, Kick, ShortRangeAccel
    pairs = []
    with torch.no_grad():
        q = torch.zeros_like(x)
        a = ShortRangeAccel.apply(x, sr, 64)
        pairs.append(sr.stats().pairs_last)
        if states is not None:
            states.append(x.clone())
        for _ in range(n_steps):
            q = Kick.apply(q, a, sr, 0.5 * dt)
            x = Drift.apply(x, q, sr, dt)
            a = ShortRangeAccel.apply(x, sr, 64)
            pairs.append(sr.stats().pairs_last)
            if states is not None:
                states.append(x.clone())
            q = Kick.apply(q, a, sr, 0.5 * dt)
    return x, pairs


def _near_cutoff(states, k, x_r, margin):
    """Does particle k have a partner within `margin` of the cutoff anywhere on the trajectory?"""
    for x in states:
        d = x - x[:, k:k + 1]
        d = d - torch.round(d)
        r = torch.sqrt((d * d).sum(dim=0))
        if float(torch.abs(r - x_r).min()) < margin:
            return True
    return False


def test_leapfrog_gradient_vs_finite_differences():
    """The 128^3 differentiable configuration: FP64 adjoint through the
    checkpointed 16-step leapfrog vs central finite differences (h = 1e-6).
    Coordinates whose +/- runs change the interacting-pair set somewhere along
    the trajectory (a pair crossing the cutoff, where the force jumps) are
    re-drawn."""
    w = synth.workload("n2m_leapfrog")
    pos = synth.workload_positions(w)
    n = w.n
    wts_np = np.stack([synth.uniform(n, 9, k * n, -1, 1) for k in range(3)])
    with ShortRange.from_workload(w) as sr:
        x_base = torch.from_numpy(pos).cuda()
        wts = torch.from_numpy(wts_np).cuda()
        acc0 = short_range_accel(x_base, sr, 64)
        dt = _dt(acc0.cpu().numpy(), w.eps)
        x0 = x_base.clone().requires_grad_(True)
        x16, _ = leapfrog(x0, torch.zeros_like(x0), sr, dt, 16, 4, precision=64)
        (x16 * wts).sum().backward()
        grad = x0.grad.cpu().numpy()
        states = []
        x16_ref, _ = _trajectory(x_base.clone(), sr, dt, 16, states)
        assert torch.equal(x16_ref, x16.detach()), "checkpointed and plain trajectories differ"
        rng = np.random.default_rng(1)
        h = 1e-6
        errs = []
        force_part = []
        for _ in range(40):
            if len(errs) >= 10:
                break
            k = int(rng.integers(n))
            d = int(rng.integers(3))
            if _near_cutoff(states, k, w.x_r, 4 * h):
                continue  # a pair of k could cross x_r between the +/- runs
            ends, prs = [], []
            for s in (+1, -1):
                xp = x_base.clone()
                xp[d, k] += s * h
                xe, pc = _trajectory(xp, sr, dt, 16)
                ends.append(xe)
                prs.append(pc)
            if prs[0] != prs[1]:
                continue
            # (L+ - L-) from the trajectory difference (no cancellation of the large sums)
            dx = ends[0] - ends[1]
            fd = float((dx * wts).sum()) / (2 * h)
            g = grad[d, k]
            errs.append(abs(fd - g) / max(abs(g), 1e-30))
            force_part.append(abs(g - wts_np[d, k]) / max(abs(g), 1e-30))
        errs = np.array(errs)
        print("dt", dt, "FD relative errors:", errs, "force part of the gradient:", np.array(force_part))
        assert len(errs) >= 8
        assert errs.max() <= 1e-6, errs
