"""The slab decomposition's host logic and exchange (paper_2112_01508_gb300/slabs.py)
on CPU: balancing, the exchange through emulated ranks and through two gloo ranks.
The tile columns come from the oracle's subtile ids (standing in for the
library's sort) and the forces from the oracle: each rank's forces on its own
particles, with its halo as extra suppliers, must reproduce the whole-box
oracle (Section 2.1.2 "Parallelisation", Section 2.1.3 "Tiles")."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
import synth
from paper_2112_01508_gb300.slabs import (LocalFabric, SlabExchange, column_offsets, column_weights,
                                          slab_bounds)

W = synth.workload("n32k")
N_T = int(np.floor(1.0 / W.x_r))
NSUB3 = W.n_sub ** 3


def test_slab_bounds_cover_and_balance():
    rng = np.random.default_rng(0)
    w = rng.random(45) ** 4 * 100
    for k in (1, 2, 3, 7, 22):
        for mw in (1, 2):
            b = slab_bounds(w, k, mw)
            assert b[0] == 0 and b[-1] == 45 and len(b) == k + 1
            assert all(b1 - b0 >= mw for b0, b1 in zip(b, b[1:]))
            parts = [w[b0:b1].sum() for b0, b1 in zip(b, b[1:])]
            if mw == 1:
                # no slab exceeds its share by more than the largest single column
                assert max(parts) <= w.sum() / k + w.max() + 1e-9
    with pytest.raises(ValueError):
        slab_bounds(w, 23, 2)


def test_balancing_follows_clustered_work():
    w = np.ones(20)
    w[3] = 200.0  # one heavy column
    b = slab_bounds(w, 4)
    j = next(i for i in range(4) if b[i] <= 3 < b[i + 1])
    assert b[j + 1] - b[j] <= 2


def test_column_offsets_and_weights_from_tile_offsets():
    n_t = 5
    counts = np.arange(n_t ** 3) % 7
    toff = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    col = column_offsets(torch.from_numpy(toff), n_t)
    per_col = counts.reshape(n_t, n_t * n_t)
    assert col == [0] + list(np.cumsum(per_col.sum(axis=1)))
    np.testing.assert_array_equal(column_weights(toff, n_t), (per_col.astype(float) ** 2).sum(axis=1))


def _columns(pos):
    """Tile column along x of every particle, from the oracle's subtile ids."""
    return oracle.subtile_ids(pos, N_T, W.n_sub) // (N_T * N_T * NSUB3)


def _sorted_rank_arrays(pos, ids):
    """The rank's particles in tile order (a stable sort of the oracle's ids) as torch
    CPU tensors [pos, ids], and the column offsets of that order."""
    sid = oracle.subtile_ids(pos, N_T, W.n_sub)
    order = np.argsort(sid, kind="stable")
    cols = sid[order] // (N_T * N_T * NSUB3)
    col_off = [int(v) for v in np.searchsorted(cols, np.arange(N_T + 1), side="left")]
    arrays = [torch.from_numpy(np.ascontiguousarray(pos[:, order])), torch.from_numpy(ids[order])]
    return arrays, col_off


def _moved_set(n, seed, step):
    """n particles of the 32^3 recipe at P0 and displaced by up to `step` (P1, wrapped)."""
    full = synth.workload_positions(W)
    idx = np.random.default_rng(seed).choice(W.n, size=n, replace=False)
    p0 = np.ascontiguousarray(full[:, idx])
    p1 = p0 + np.random.default_rng(seed + 1).uniform(-step, step, size=p0.shape)
    p1 -= np.floor(p1)
    p1[p1 >= 1.0] = 0.0
    return p0, p1


def _bounds(p0, k):
    cols = _columns(p0)
    tiles = oracle.subtile_ids(p0, N_T, W.n_sub) // NSUB3
    counts = np.bincount(tiles, minlength=N_T ** 3).astype(float).reshape(N_T, N_T * N_T)
    return slab_bounds((counts ** 2).sum(axis=1), k, 2), cols


def _check_rank(ex, own, halo, p1, ref, expect_pairs=None):
    """Own particles lie in the slab; the halo is exactly columns t0-1 and t1; the
    forces on the own particles equal the whole-box oracle's."""
    c1 = _columns(p1)
    ids = own[1].numpy()
    own_pos = own[0].numpy()
    np.testing.assert_array_equal(own_pos, p1[:, ids])
    assert np.all((c1[ids] >= ex.t0) & (c1[ids] < ex.t1))
    halo_np = halo.numpy()
    if ex.world > 1:
        want = np.flatnonzero((c1 == ex.left_col) | (c1 == ex.right_col))
        got = np.lexsort(halo_np)
        exp = p1[:, want]
        np.testing.assert_array_equal(halo_np[:, got], exp[:, np.lexsort(exp)])
    comb = np.ascontiguousarray(np.concatenate([own_pos, halo_np], axis=1))
    flag = np.zeros(comb.shape[1], np.int8)
    flag[:len(ids)] = 1
    acc, pairs = oracle.sr_accel(comb, W.x_s, W.x_r, W.G_m, "bspline", W.eps, rung=flag, rung_min=1)
    err = np.sqrt(((acc[:, :len(ids)] - ref[:, ids]) ** 2).sum() / (ref[:, ids] ** 2).sum())
    assert err <= 1e-13
    return len(ids), pairs


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_exchange_with_emulated_ranks_reproduces_the_whole_box(k):
    n = 8192
    p0, p1 = _moved_set(n, 3, 0.5 / N_T)  # at most half a column per coordinate
    bounds, c0 = _bounds(p0, k)
    ref, ref_pairs = oracle.sr_accel(p1, W.x_s, W.x_r, W.G_m, "bspline", W.eps)
    exs = [SlabExchange(N_T, bounds, r, k) for r in range(k)]
    outs = []
    for ex in exs:
        mine = np.flatnonzero((c0 >= ex.t0) & (c0 < ex.t1))   # owned at P0, positions now at P1
        arrays, col_off = _sorted_rank_arrays(p1[:, mine], mine.astype(np.int64))
        outs.append(ex.prepare(arrays, col_off))
    swapped = LocalFabric.swap_all(exs, outs)
    seen, pairs = [], 0
    for ex, out, (fl, fr) in zip(exs, outs, swapped):
        own, halo = ex.finish(out, fl, fr)
        seen.append(own[1].numpy())
        pairs += _check_rank(ex, own, halo, p1, ref)[1]
    allids = np.concatenate(seen)
    np.testing.assert_array_equal(np.sort(allids), np.arange(n))  # every particle owned once
    assert pairs == ref_pairs
    if k > 1:  # some particles changed owner
        moved = sum(int((~np.isin(own_ids, np.flatnonzero((c0 >= ex.t0) & (c0 < ex.t1)))).sum())
                    for own_ids, ex in zip(seen, exs))
        assert moved > 0


def test_exchange_rejects_jumps_over_a_column():
    n = 4096
    p0, _ = _moved_set(n, 4, 0.0)
    bounds, c0 = _bounds(p0, 3)
    ex = SlabExchange(N_T, bounds, 1, 3)
    p1 = p0.copy()
    p1[0] = (p1[0] + 2.5 / N_T) % 1.0  # everything moves by 2.5 columns
    mine = np.flatnonzero((c0 >= ex.t0) & (c0 < ex.t1))
    arrays, col_off = _sorted_rank_arrays(p1[:, mine], mine.astype(np.int64))
    with pytest.raises(RuntimeError):
        ex.prepare(arrays, col_off)
    with pytest.raises(ValueError):
        SlabExchange(N_T, [0, 1, N_T], 0, 2)  # a one-column slab


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2112_01508_gb300.slabs import DistTransport
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 8192
        p0, p1 = _moved_set(n, 5, 0.5 / N_T)
        bounds, c0 = _bounds(p0, world)
        ref, ref_pairs = oracle.sr_accel(p1, W.x_s, W.x_r, W.G_m, "bspline", W.eps)
        ex = SlabExchange(N_T, bounds, rank, world)
        mine = np.flatnonzero((c0 >= ex.t0) & (c0 < ex.t1))
        arrays, col_off = _sorted_rank_arrays(p1[:, mine], mine.astype(np.int64))
        out = ex.prepare(arrays, col_off)
        fl, fr = DistTransport().swap(ex, out)
        own, halo = ex.finish(out, fl, fr)
        n_own, pairs = _check_rank(ex, own, halo, p1, ref)
        ids = [None] * world
        dist.all_gather_object(ids, own[1].numpy().tolist())
        tot = torch.tensor([pairs], dtype=torch.int64)
        dist.all_reduce(tot)
        allids = np.sort(np.concatenate([np.asarray(v) for v in ids]))
        q.put((rank, bool(np.array_equal(allids, np.arange(n))), int(tot.item()) == ref_pairs, n_own))
    except Exception as e:  # report instead of hanging the other rank's assertions
        q.put((rank, False, repr(e), 0))
        raise
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_over_gloo_ranks_reproduces_the_whole_box(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    res = sorted(q.get(timeout=10) for _ in range(world))
    for p in procs:
        assert p.exitcode == 0
    for rank, partition_ok, pairs_ok, n_own in res:
        assert partition_ok is True and pairs_ok is True, (rank, partition_ok, pairs_ok)
        assert n_own > 0
