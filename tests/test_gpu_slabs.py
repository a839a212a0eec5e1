"""Slab ranks emulated on one GPU (paper_2112_01508_gb300/slabs.py through the
library's sort, tile offsets and forces) give the whole-box short-range force,
also over steps in which particles migrate between slabs."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2112_01508_gb300 import ShortRange
from paper_2112_01508_gb300.slabs import LocalFabric, SlabExchange, SlabRank, emulated_forces, initial_split
from tests._gpu_helpers import gpu_forces, rel_rms

pytestmark = pytest.mark.gpu


def _maker(w):
    def make(n):
        return ShortRange(max(n, 1), w.x_s, w.x_r, w.G_m, softening="bspline", eps=w.eps, n_sub=w.n_sub)
    return make


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_slabs_match_oracle_32k(k):
    w = synth.workload("n32k")
    pos = synth.workload_positions(w)
    ref, pairs = oracle.sr_accel(pos, w.x_s, w.x_r, w.G_m, "bspline", w.eps)
    p = torch.from_numpy(pos).cuda()
    for prec, tol in ((64, 1e-12), (32, 1e-5)):
        acc, npairs, bounds = emulated_forces(p, _maker(w), k, prec)
        assert len(bounds) == k + 1
        assert rel_rms(acc.double().cpu().numpy(), ref) <= tol
        if prec == 64:
            assert npairs == pairs
        else:
            assert abs(npairs - pairs) <= max(2, 1e-6 * pairs)


def test_slabs_balance_and_match_whole_box_128():
    w = synth.workload("n2m")
    pos = synth.workload_positions(w)
    whole = gpu_forces(pos, w.x_s, w.x_r, w.G_m, "bspline", w.eps, precision=64, n_sub=w.n_sub)
    p = torch.from_numpy(pos).cuda()
    acc, npairs, bounds = emulated_forces(p, _maker(w), 4, 64)
    assert npairs == whole["pairs"]
    assert rel_rms(acc.cpu().numpy(), whole["acc"]) <= 1e-13
    widths = [b1 - b0 for b0, b1 in zip(bounds, bounds[1:])]
    assert sum(widths) == int(np.floor(1.0 / w.x_r)) and min(widths) >= 2
    print("slab widths", widths)


def test_slab_steps_with_migration_match_the_oracle():
    """Three ranks, three steps of exchange -> forces -> rungs + kick + drift of the own
    particles: every step's forces equal the whole-box oracle's on the same positions,
    every particle is owned by exactly one rank, and particles change owner."""
    w = synth.workload("n32k")
    n, k = w.n, 3
    pos = torch.from_numpy(synth.workload_positions(w)).cuda()
    ids = torch.arange(n, dtype=torch.int64, device="cuda")
    mom = (0.3 * torch.randn((3, n), generator=torch.Generator().manual_seed(3), dtype=torch.float64)).cuda()
    rung = torch.zeros(n, dtype=torch.int8, device="cuda")
    make = _maker(w)
    with make(n) as full:
        bounds, parts = initial_split(full, pos, [mom, rung, ids], k)
        n_t = full.stats_geometry()[0]
    exs = [SlabExchange(n_t, bounds, r, k) for r in range(k)]
    ranks = [SlabRank(make, ex) for ex in exs]
    dt, eta = 0.03, 0.025
    kf = [dt / 2 ** l for l in range(8)]
    owner0 = None
    changed = 0
    for step in range(3):
        outs = [rk.ex.prepare(arr, rk.sort_own(arr)) for rk, arr in zip(ranks, parts)]
        swapped = LocalFabric.swap_all(exs, outs)
        allpos = np.empty((3, n))
        accs = np.empty((3, n))
        owner = np.full(n, -1)
        pairs = 0
        new_parts = []
        for r, (rk, out, (fl, fr)) in enumerate(zip(ranks, outs, swapped)):
            own, halo = rk.ex.finish(out, fl, fr)
            a, p = rk.forces(own[0], halo, 64)
            pairs += p
            oid = own[3].cpu().numpy()
            assert np.all(owner[oid] == -1)
            owner[oid] = r
            allpos[:, oid] = own[0].cpu().numpy()
            accs[:, oid] = a.cpu().numpy()
            rk.kick_drift(own, a, dt, eta, w.eps, kf, dt)
            new_parts.append(own)
        assert np.all(owner >= 0)
        ref, ref_pairs = oracle.sr_accel(allpos, w.x_s, w.x_r, w.G_m, "bspline", w.eps)
        assert pairs == ref_pairs
        assert rel_rms(accs, ref) <= 1e-12
        if owner0 is not None:
            changed += int((owner != owner0).sum())
        owner0 = owner
        parts = new_parts
    assert changed > 0
    for rk in ranks:
        rk.close()


@pytest.mark.parametrize("n_subs", [(1, 2, 3), (3, 1, 2), (2, 4, 1)])
def test_mixed_per_region_subtiles_match_the_oracle(n_subs):
    """Each slab region with its own subtiles per tile (Section 2.1.3, "Subtiles": the
    decomposition of a domain is its own): the forces still equal the oracle's."""
    w = synth.workload("n32k")
    pos = synth.workload_positions(w)
    ref, pairs = oracle.sr_accel(pos, w.x_s, w.x_r, w.G_m, "bspline", w.eps)
    p = torch.from_numpy(pos).cuda()
    for prec, tol in ((64, 1e-12), (32, 1e-5)):
        acc, npairs, _ = emulated_forces(p, _maker(w), len(n_subs), prec, n_subs=list(n_subs))
        assert rel_rms(acc.double().cpu().numpy(), ref) <= tol
        if prec == 64:
            assert npairs == pairs


def test_region_refiner_refines_each_region_by_its_own_timing():
    """The timed trial rule per region: every region starts at one subtile per tile and
    tries one more every `interval` force calls; the kept decompositions may differ
    between regions, and the forces with the final map still equal the oracle's."""
    from paper_2112_01508_gb300.refine import RegionRefiner
    from paper_2112_01508_gb300.slabs import EmulatedSlabs
    w = synth.workload("n32k")
    pos = synth.workload_positions(w)
    ref, _ = oracle.sr_accel(pos, w.x_s, w.x_r, w.G_m, "bspline", w.eps)
    em = EmulatedSlabs(torch.from_numpy(pos).cuda(), _maker(w), 3, n_subs=[1, 1, 1])
    rr = RegionRefiner(em.ranks, interval=4, max_sub=3)
    for _ in range(16):
        rr.before_sort()
        res = em.forces(32)
        rr.after_forces()
    assert all(log.trials >= 1 for log in rr.logs)
    print("per-region subtiles", rr.current, [[e[1:] for e in log.events] for log in rr.logs])
    rr.before_sort()
    acc, _ = em.gather(em.forces(64))
    assert rel_rms(acc.cpu().numpy(), ref) <= 1e-12
    em.close()
