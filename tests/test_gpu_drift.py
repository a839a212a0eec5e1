"""Forces, adjoint and work lists on positions drifted since the last sort
(the sort is reused, the traversal reach widened by the recorded drift)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2112_01508_gb300 import ShortRange
from paper_2112_01508_gb300 import _native as nat
from tests._gpu_helpers import rel_rms

pytestmark = pytest.mark.gpu

W = synth.workload("n32k")


def _drifted(n_drifts, speed, seed=2):
    """Sorted n32k positions drifted n_drifts times (no sort in between)."""
    pos = synth.workload_positions(W)
    rng = np.random.default_rng(seed)
    mom = rng.normal(size=pos.shape) * speed
    return pos, mom


@pytest.mark.parametrize("n_drifts,speed", [(1, 0.004), (4, 0.004), (8, 0.002)])
def test_forces_and_vjp_after_drifts(n_drifts, speed):
    pos, mom_np = _drifted(n_drifts, speed)
    with ShortRange.from_workload(W) as sr:
        p = torch.from_numpy(pos.copy()).cuda()
        q = torch.from_numpy(mom_np).cuda()
        rung = torch.from_numpy(np.random.default_rng(5).integers(0, 3, W.n).astype(np.int8)).cuda()
        sr.sort(p, carry=[q, rung])
        for _ in range(n_drifts):
            sr.drift(p, q, 1.0)  # displacement |q| per drift: up to ~0.02 of a 0.044 subtile
        x = p.cpu().numpy()
        # some particles crossed the periodic boundary since the sort
        sr.build_pairs()
        a64 = sr.forces(p, 64)
        st = sr.stats()
        a32 = sr.forces(p, 32)
        abar = torch.from_numpy(np.random.default_rng(9).normal(size=(3, W.n))).cuda()
        xb = sr.vjp(p, abar, 64)
        sr.build_pairs(rung, 1)
        a_act = torch.full((3, W.n), float("nan"), dtype=torch.float64, device="cuda")
        sr.forces(p, 64, a_act)
        sr.sync()
    ref, pairs = oracle.sr_accel(x, W.x_s, W.x_r, W.G_m, "bspline", W.eps)
    assert st.pairs_last == pairs
    assert rel_rms(a64.cpu().numpy(), ref) <= 1e-12
    assert rel_rms(a32.cpu().numpy(), ref) <= 1e-5
    xref = oracle.sr_vjp(x, abar.cpu().numpy(), W.x_s, W.x_r, W.G_m, "bspline", W.eps)
    assert rel_rms(xb.cpu().numpy(), xref) <= 1e-12
    act = rung.cpu().numpy() >= 1
    ref_act, _ = oracle.sr_accel(x, W.x_s, W.x_r, W.G_m, "bspline", W.eps, rung=rung.cpu().numpy(), rung_min=1)
    got = a_act.cpu().numpy()
    assert rel_rms(got[:, act], ref_act[:, act]) <= 1e-12
    assert np.all(np.isnan(got[:, ~act]))


def test_positions_crossing_the_box_edge():
    # particles near x = 0 and x = L drift across the periodic boundary
    rng = np.random.default_rng(1)
    n = 6000
    pos = rng.random((3, n))
    pos[0, :1000] = rng.random(1000) * 0.01
    pos[0, 1000:2000] = 1.0 - rng.random(1000) * 0.01
    mom = np.zeros((3, n))
    mom[0, :1000] = -0.02
    mom[0, 1000:2000] = 0.02
    x_r = 0.1
    with ShortRange(n, x_r / 4.5, x_r, 1.0 / n, softening="plummer", eps=0.002, n_sub=2) as sr:
        p = torch.from_numpy(pos.copy()).cuda()
        q = torch.from_numpy(mom).cuda()
        sr.sort(p, carry=[q])
        sr.drift(p, q, 1.0)
        sr.build_pairs()
        a64 = sr.forces(p, 64)
        a32 = sr.forces(p, 32)
        st = sr.stats()
        sr.sync()
        x = p.cpu().numpy()
    ref, pairs = oracle.sr_accel(x, x_r / 4.5, x_r, 1.0 / n, "plummer", 0.002)
    assert st.pairs_last == pairs
    assert rel_rms(a64.cpu().numpy(), ref) <= 1e-12
    assert rel_rms(a32.cpu().numpy(), ref) <= 1e-5


def test_sort_dropped_after_64_drifts():
    n = 512
    with ShortRange(n, W.x_s, W.x_r, W.G_m, softening="bspline", eps=W.eps) as sr:
        p = torch.rand((3, n), dtype=torch.float64, device="cuda")
        q = torch.zeros_like(p)
        sr.sort(p)
        for _ in range(64):
            sr.drift(p, q, 1.0)
        sr.build_pairs()  # still usable
        sr.drift(p, q, 1.0)
        with pytest.raises(nat.P3MError) as e:
            sr.build_pairs()
        assert e.value.status == nat.P3M_ERR_STATE
        sr.sort(p)
        sr.build_pairs()
        sr.sync()


def test_excessive_drift_is_reported():
    n = 2048
    with ShortRange(n, W.x_s, W.x_r, W.G_m, softening="bspline", eps=W.eps) as sr:
        p = torch.rand((3, n), dtype=torch.float64, device="cuda")
        q = torch.full_like(p, 0.2)  # |q| = 0.35 per drift: x_r + 2 drift > L/2
        sr.sort(p)
        sr.drift(p, q, 1.0)
        sr.build_pairs()
        sr.forces(p, 32)
        with pytest.raises(nat.P3MError) as e:
            sr.sync()
        assert e.value.status == nat.P3M_ERR_STATE
