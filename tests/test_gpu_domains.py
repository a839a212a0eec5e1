"""Slab domains emulated on one GPU give the whole-box short-range force."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2112_01508_gb300.domains import emulated_forces
from tests._gpu_helpers import gpu_forces, rel_rms

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_domains_match_oracle_32k(k):
    w = synth.workload("n32k")
    pos = synth.workload_positions(w)
    ref, pairs = oracle.sr_accel(pos, w.x_s, w.x_r, w.G_m, "bspline", w.eps)
    p = torch.from_numpy(pos).cuda()
    for prec, tol in ((64, 1e-12), (32, 1e-5)):
        acc, npairs, doms = emulated_forces(p, w.x_s, w.x_r, w.G_m, k, "bspline", w.eps, w.n_sub, prec)
        assert len(doms) == k
        assert rel_rms(acc.double().cpu().numpy(), ref) <= tol
        if prec == 64:
            assert npairs == pairs


def test_domains_balance_and_match_whole_box_128():
    w = synth.workload("n2m")
    pos = synth.workload_positions(w)
    whole = gpu_forces(pos, w.x_s, w.x_r, w.G_m, "bspline", w.eps, precision=64, n_sub=w.n_sub)
    p = torch.from_numpy(pos).cuda()
    acc, npairs, doms = emulated_forces(p, w.x_s, w.x_r, w.G_m, 4, "bspline", w.eps, w.n_sub, 64)
    assert npairs == whole["pairs"]
    assert rel_rms(acc.cpu().numpy(), whole["acc"]) <= 1e-13
    # the balanced slabs differ in width (the work estimate follows the clustering)
    widths = [d.tiles[1] - d.tiles[0] for d in doms]
    assert sum(widths) == int(np.floor(1.0 / w.x_r))
    print("slab widths", widths, "particles", [len(d.local) for d in doms])
