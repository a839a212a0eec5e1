"""GPU checks of p3m_sr_set_subtiles and the temporal subtile refinement."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2112_01508_gb300 import ShortRange
from paper_2112_01508_gb300 import _native as nat
from paper_2112_01508_gb300.refine import SubtileRefiner
from tests._gpu_helpers import rel_rms

pytestmark = pytest.mark.gpu

W = synth.workload("n32k")
FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def n32k():
    pos = synth.workload_positions(W)
    return pos, oracle.sr_accel(pos, W.x_s, W.x_r, W.G_m, "bspline", W.eps)


def _forces(sr, pos_np, prec):
    """Sort a fresh device copy of pos_np, build, forces; accelerations in pos_np's order."""
    p = torch.from_numpy(np.ascontiguousarray(pos_np)).cuda()
    perm = torch.empty(sr.n, dtype=torch.int32, device=p.device)
    sr.sort(p, perm_out=perm)
    sr.build_pairs()
    out = sr.forces(p, prec)
    st = sr.stats()
    acc = np.empty((3, sr.n))
    acc[:, perm.cpu().numpy().astype(np.int64)] = out.cpu().numpy()
    return acc, st


def test_set_subtiles_changes_nothing_but_the_decomposition(n32k):
    pos, (ref, pairs) = n32k
    with ShortRange.from_workload(W, n_sub=1) as sr:
        for ns in [(1, 1, 1), (3, 3, 3), (2, 3, 1), (5, 5, 5), (1, 1, 1)]:
            sr.set_subtiles(ns)
            with pytest.raises(nat.P3MError) as e:
                sr.build_pairs()  # the sort state is dropped
            assert e.value.status == nat.P3M_ERR_STATE
            for prec, tol in ((64, FP64_TOL), (32, FP32_TOL)):
                acc, st = _forces(sr, pos, prec)
                assert tuple(st.n_sub) == ns
                assert rel_rms(acc, ref) <= tol
                if prec == 64:
                    assert st.pairs_last == pairs
        # invalid request: error, and the decomposition in force is unchanged
        with pytest.raises(nat.P3MError) as e:
            sr.set_subtiles((17, 1, 1))
        assert e.value.status == nat.P3M_ERR_INVALID
        acc, st = _forces(sr, pos, 64)
        assert tuple(st.n_sub) == (1, 1, 1)
        assert rel_rms(acc, ref) <= FP64_TOL


def test_refiner_in_a_step_loop(n32k):
    pos, _ = n32k
    p = torch.from_numpy(pos.copy()).cuda()
    mom = torch.zeros_like(p)
    acc = torch.zeros((3, W.n), dtype=torch.float32, device="cuda")
    with ShortRange.from_workload(W, n_sub=1) as sr:
        ref = SubtileRefiner(sr, interval=4, max_sub=4)
        for _ in range(24):
            ref.before_sort()
            sr.sort(p, carry=[mom])
            sr.build_pairs()
            sr.forces(p, 32, acc)
            ref.after_forces()
            sr.kick(mom, acc, [1e-6])
            sr.drift(p, mom, 1e-6)
        sr.sync()
        assert ref.log.trials >= 3
        assert tuple(sr.n_sub) in {ref.current, tuple(v + 1 for v in ref.current)}
        # the state reached through the switches still gives the oracle's forces
        pos_now = p.cpu().numpy()
        r, pairs = oracle.sr_accel(pos_now, W.x_s, W.x_r, W.G_m, "bspline", W.eps)
        ref.before_sort()
        got, st = _forces(sr, pos_now, 64)
        assert st.pairs_last == pairs
        assert rel_rms(got, r) <= FP64_TOL
