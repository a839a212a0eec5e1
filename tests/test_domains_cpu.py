"""Host logic of the slab decomposition (paper_2112_01508_gb300/domains.py), on CPU."""
import numpy as np
import pytest

import synth
from paper_2112_01508_gb300.domains import column_weights, decompose, slab_bounds, tile_indices


def test_slab_bounds_cover_and_balance():
    rng = np.random.default_rng(0)
    w = rng.random(45) ** 4 * 100
    for k in (1, 2, 3, 7, 45):
        b = slab_bounds(w, k)
        assert b[0] == 0 and b[-1] == 45 and len(b) == k + 1
        assert all(b1 > b0 for b0, b1 in zip(b, b[1:]))
        parts = [w[b0:b1].sum() for b0, b1 in zip(b, b[1:])]
        if k < 45:
            # no slab exceeds its share by more than the largest single column
            assert max(parts) <= w.sum() / k + w.max() + 1e-9
    with pytest.raises(ValueError):
        slab_bounds(w, 46)


def test_balancing_follows_clustered_work():
    w = np.ones(20)
    w[3] = 200.0  # one heavy column
    b = slab_bounds(w, 4)
    # the heavy column sits in a slab of its own or nearly so
    j = next(i for i in range(4) if b[i] <= 3 < b[i + 1])
    assert b[j + 1] - b[j] <= 2


def test_decomposition_partitions_and_halos():
    w = synth.workload("n32k")
    pos = synth.workload_positions(w)
    n_t = int(np.floor(1.0 / w.x_r))
    tiles = tile_indices(pos, n_t)
    cw = column_weights(tiles, n_t)
    assert cw.shape == (n_t,) and cw.sum() > 0
    for k in (1, 2, 3, 5):
        doms = decompose(pos, n_t, k)
        allloc = np.concatenate([d.local for d in doms])
        assert np.array_equal(np.sort(allloc), np.arange(w.n))  # every particle in one slab
        for d in doms:
            t0, t1 = d.tiles
            assert np.all((tiles[0, d.local] >= t0) & (tiles[0, d.local] < t1))
            assert len(np.intersect1d(d.local, d.halo)) == 0
            if k > 1:
                expect = {(t0 - 1) % n_t, t1 % n_t} - set(range(t0, t1))
                assert set(np.unique(tiles[0, d.halo])) <= expect
                # every particle of those columns is in the halo
                want = np.flatnonzero(np.isin(tiles[0], list(expect)))
                assert np.array_equal(np.sort(d.halo), want)
