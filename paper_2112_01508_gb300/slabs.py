"""Slab decomposition of the periodic box over ranks, for the short-range force
(the paper's domains, Section 2.1.2 "Parallelisation", and its tile-level
pairing of neighbouring domains, Section 2.1.3 "Tiles").

Each rank owns a slab of whole tile columns [t0, t1) along x.  Tiles are at
least x_r wide, so the receivers of a slab need as suppliers only the
particles of one tile column on each side (the halo).  One exchange per force
evaluation, with the two neighbouring ranks only, moves

  * the emigrants: own particles that drifted into a neighbour's edge column
    (at most one column per step), which change owner, and
  * the halo: the positions of the slab's two edge columns, which the
    neighbours need as suppliers.

A rank's halo is then the neighbour's edge column plus its own emigrants into
that column (every slab is at least two columns wide, so a column next to a
slab holds no immigrant from further away).  The rank sorts its particles plus
halo in its own memory and computes the forces of its own particles only (the
one-sided kernel: no partial sums are sent back, unlike the paper's momentum
send-back).  Slab boundaries follow the prefix of a per-column work estimate,
the sum over the column's tiles of (particles per tile)^2 -- a tile's pair
count up to a constant -- which addresses the load imbalance under clustering
that the paper names as its scheme's main weakness.

The exchange runs through a transport: ``DistTransport`` (torch.distributed
point-to-point sends, NCCL between GPUs or gloo on CPU) or ``LocalFabric``
(several ranks emulated in one process, for tests on one GPU).  Which
particles go where is read from the tile ranges of the library's sort
(``ShortRange.tile_offsets``); nothing here bins positions.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch


# ---------------------------------------------------------------------------
# Host logic: slab boundaries and the per-column work estimate.
# ---------------------------------------------------------------------------

def slab_bounds(weights, k: int, min_width: int = 1) -> list[int]:
    """Boundaries 0 = b_0 < ... < b_k = n_t of k slabs of whole columns: each slab in
    turn takes the prefix closest to an equal share of the weight still to assign
    (a heavy column then sits in a slab of its own and the rest is spread over the
    others); every slab keeps at least `min_width` columns."""
    w = np.asarray(weights, dtype=np.float64)
    n_t = len(w)
    if not 1 <= k or k * min_width > n_t:
        raise ValueError("need 1 <= k and k * min_width <= number of tile columns")
    c = np.concatenate([[0.0], np.cumsum(w)])
    b = [0]
    for j in range(1, k):
        start = b[-1]
        target = c[start] + (c[-1] - c[start]) / (k - j + 1)
        lo, hi = start + min_width, n_t - (k - j) * min_width  # room for the slabs still to come
        t = min(max(int(np.searchsorted(c, target, side="left")), lo), hi)
        if t - 1 >= lo and abs(c[t - 1] - target) <= abs(c[t] - target):
            t -= 1
        b.append(t)
    b.append(n_t)
    return b


def column_offsets(tile_offsets, n_t: int) -> list[int]:
    """Sorted index of the first particle of every tile column along x (n_t + 1
    values), from the n_t^3 + 1 tile offsets of a sort."""
    off = tile_offsets.cpu() if isinstance(tile_offsets, torch.Tensor) else torch.as_tensor(tile_offsets)
    return [int(v) for v in off[:: n_t * n_t][: n_t + 1]]


def column_weights(tile_offsets, n_t: int) -> np.ndarray:
    """Work estimate per tile column along x: the sum over its tiles of count^2."""
    off = tile_offsets.cpu().numpy() if isinstance(tile_offsets, torch.Tensor) else np.asarray(tile_offsets)
    counts = np.diff(off.astype(np.int64)).astype(np.float64).reshape(n_t, n_t * n_t)
    return (counts ** 2).sum(axis=1)


# ---------------------------------------------------------------------------
# The exchange.
# ---------------------------------------------------------------------------

@dataclass
class Outgoing:
    """What one rank sends to each neighbour and what it keeps."""
    to_left: list        # [emigrants of every array..., halo positions]
    to_right: list
    counts_left: tuple   # (emigrants, halo particles)
    counts_right: tuple
    stay: list           # every array, the particles that stay (in sorted order)


class SlabExchange:
    """The exchange pattern of one rank: slab [t0, t1) of n_t tile columns, neighbours
    (rank - 1) and (rank + 1) modulo the number of ranks."""

    def __init__(self, n_t: int, bounds, rank: int, world: int):
        if len(bounds) != world + 1 or bounds[0] != 0 or bounds[-1] != n_t:
            raise ValueError("bounds must hold world + 1 column boundaries from 0 to n_t")
        if world > 1 and min(b1 - b0 for b0, b1 in zip(bounds, bounds[1:])) < 2:
            raise ValueError("every slab must be at least two tile columns wide")
        self.n_t, self.bounds, self.rank, self.world = n_t, list(bounds), rank, world
        self.t0, self.t1 = bounds[rank], bounds[rank + 1]
        self.left, self.right = (rank - 1) % world, (rank + 1) % world
        self.left_col, self.right_col = (self.t0 - 1) % n_t, self.t1 % n_t

    def prepare(self, arrays, col_off) -> Outgoing:
        """Split this rank's particles, sorted by tile column (the order of a sort:
        `col_off` the n_t + 1 column offsets), into those that stay, the emigrants to
        each neighbour and the halo positions each neighbour needs.  arrays[0] is the
        (3, n) positions; every array has particles on its last dimension."""
        n = arrays[0].shape[-1]
        if col_off[-1] != n:
            raise ValueError("column offsets do not match the particle count")

        def cols(c):
            return col_off[c], col_off[c + 1]
        s0, s1 = col_off[self.t0], col_off[self.t1]
        if self.world == 1:
            stay = list(arrays)
            return Outgoing([], [], (0, 0), (0, 0), stay)
        l0, l1 = cols(self.left_col)
        r0, r1 = cols(self.right_col)
        if (l1 - l0) + (r1 - r0) + (s1 - s0) != n:
            raise RuntimeError("a particle moved more than one tile column since the last exchange")
        h0 = cols(self.t0)
        h1 = cols(self.t1 - 1)
        pos = arrays[0]
        to_left = [a[..., l0:l1] for a in arrays] + [pos[..., h0[0]:h0[1]]]
        to_right = [a[..., r0:r1] for a in arrays] + [pos[..., h1[0]:h1[1]]]
        stay = [a[..., s0:s1] for a in arrays]
        return Outgoing(to_left, to_right, (l1 - l0, h0[1] - h0[0]), (r1 - r0, h1[1] - h1[0]), stay)

    def finish(self, out: Outgoing, from_left, from_right):
        """Own particles after the exchange (stayed, then immigrants from the left, then
        from the right: every array) and the halo positions (3, m): the neighbours'
        edge columns plus this rank's own emigrants into them."""
        if self.world == 1:
            empty = out.stay[0][..., :0]
            return [a.contiguous() for a in out.stay], empty.contiguous()
        m = len(out.stay)
        own = [torch.cat([out.stay[k], from_left[k], from_right[k]], dim=-1).contiguous() for k in range(m)]
        halo = torch.cat([from_left[m], out.to_left[0], from_right[m], out.to_right[0]], dim=-1).contiguous()
        return own, halo


class DistTransport:
    """Point-to-point exchange with the two neighbours through torch.distributed (NCCL
    for CUDA tensors, gloo for CPU tensors): counts first, then the payload."""

    TAG_TO_LEFT, TAG_TO_RIGHT = 11, 12

    def __init__(self, group=None):
        self.group = group

    def swap(self, ex: SlabExchange, out: Outgoing):
        import torch.distributed as dist
        if ex.world == 1:
            return [], []
        like = out.stay
        dev = like[0].device
        c_left = torch.tensor(out.counts_left, dtype=torch.int64, device=dev)
        c_right = torch.tensor(out.counts_right, dtype=torch.int64, device=dev)
        r_from_left = torch.empty(2, dtype=torch.int64, device=dev)
        r_from_right = torch.empty(2, dtype=torch.int64, device=dev)
        # a message to the left neighbour arrives there as "from the right": tags name the direction
        ops = [dist.P2POp(dist.isend, c_left, ex.left, self.group, self.TAG_TO_LEFT),
               dist.P2POp(dist.isend, c_right, ex.right, self.group, self.TAG_TO_RIGHT),
               dist.P2POp(dist.irecv, r_from_right, ex.right, self.group, self.TAG_TO_LEFT),
               dist.P2POp(dist.irecv, r_from_left, ex.left, self.group, self.TAG_TO_RIGHT)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        n_fl, n_fr = [int(v) for v in r_from_left.tolist()], [int(v) for v in r_from_right.tolist()]

        def buffers(counts):
            bufs = [torch.empty(tuple(a.shape[:-1]) + (counts[0],), dtype=a.dtype, device=dev) for a in like]
            bufs.append(torch.empty(tuple(like[0].shape[:-1]) + (counts[1],), dtype=like[0].dtype, device=dev))
            return bufs
        from_left, from_right = buffers(n_fl), buffers(n_fr)
        ops = []
        for t in out.to_left:
            if t.shape[-1]:
                ops.append(dist.P2POp(dist.isend, t.contiguous(), ex.left, self.group, self.TAG_TO_LEFT))
        for t in out.to_right:
            if t.shape[-1]:
                ops.append(dist.P2POp(dist.isend, t.contiguous(), ex.right, self.group, self.TAG_TO_RIGHT))
        for t in from_right:
            if t.shape[-1]:
                ops.append(dist.P2POp(dist.irecv, t, ex.right, self.group, self.TAG_TO_LEFT))
        for t in from_left:
            if t.shape[-1]:
                ops.append(dist.P2POp(dist.irecv, t, ex.left, self.group, self.TAG_TO_RIGHT))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        return from_left, from_right


class LocalFabric:
    """Several ranks emulated in one process: every rank's outgoing lists are handed
    to its neighbours directly."""

    @staticmethod
    def swap_all(exchanges, outs):
        res = []
        for ex, out in zip(exchanges, outs):
            if ex.world == 1:
                res.append(([], []))
                continue
            from_left = [t.clone() for t in outs[ex.left].to_right]
            from_right = [t.clone() for t in outs[ex.right].to_left]
            res.append((from_left, from_right))
        return res


# ---------------------------------------------------------------------------
# One rank on its GPU: contexts with room for migration.
# ---------------------------------------------------------------------------

class SlabRank:
    """The short-range computation of one rank: a context for its own particles (to
    find their tile columns) and one for own particles plus halo (the forces).
    Contexts are created with room to spare and grow when a count exceeds it."""

    def __init__(self, make_context, exchange: SlabExchange, headroom: float = 1.25, n_sub=None):
        self.make = make_context
        self.ex = exchange
        self.headroom = headroom
        self.sr_own = None
        self.sr_all = None
        # subtiles per tile of this slab's force context (None: the context's default); a
        # slab may use its own decomposition (Section 2.1.3, "Subtiles": per domain)
        self.n_sub = None if n_sub is None else ((n_sub,) * 3 if isinstance(n_sub, int) else tuple(n_sub))

    def _ctx(self, which: str, n: int):
        sr = getattr(self, which)
        if sr is None or sr.capacity < n:
            if sr is not None:
                sr.close()
            sr = self.make(max(int(n * self.headroom), 1))
            setattr(self, which, sr)
        if which == "sr_all" and self.n_sub is not None and tuple(sr.n_sub) != self.n_sub:
            sr.set_subtiles(self.n_sub)
        sr.set_count(n)
        return sr

    def set_subtiles(self, n_sub):
        """Subtiles per tile of this slab's force context from its next force call on."""
        self.n_sub = (n_sub,) * 3 if isinstance(n_sub, int) else tuple(n_sub)

    def stats(self):
        """Counters of the force context (its last force call)."""
        return self.sr_all.stats()

    def sort_own(self, arrays):
        """Sort the own particles into tiles (every array carried); returns the column offsets."""
        sr = self._ctx("sr_own", arrays[0].shape[-1])
        sr.sort(arrays[0], carry=list(arrays[1:]))
        return column_offsets(sr.tile_offsets(), self.ex.n_t)

    def forces(self, own_pos: torch.Tensor, halo_pos: torch.Tensor, precision: int = 32):
        """Accelerations (3, n_own) of the own particles, in their order, with the halo as
        extra suppliers; also returns the interacting pairs met."""
        n_own, n_halo = own_pos.shape[1], halo_pos.shape[1]
        sr = self._ctx("sr_all", n_own + n_halo)
        comb = torch.cat([own_pos, halo_pos], dim=1).contiguous()
        flag = torch.zeros(n_own + n_halo, dtype=torch.int8, device=comb.device)
        flag[:n_own] = 1
        sr.sort(comb, carry=[flag])
        sr.build_pairs(flag, 1)
        acc = sr.forces(comb, precision)
        pairs = sr.stats().pairs_last
        return sr.unpermute(acc)[:, :n_own].contiguous(), pairs

    def kick_drift(self, own, acc: torch.Tensor, dt: float, eta: float, eps: float, kick_factor,
                   drift_factor: float):
        """Rungs, kick and drift of the own particles (p3m_sr_kick_drift); own = [pos (3, n),
        mom (3, n), rung (n), ...] in the order of `acc`."""
        sr = self._ctx("sr_own", own[0].shape[-1])
        sr.kick_drift(own[0], own[1], acc, own[2], dt, eta, eps, kick_factor, drift_factor)

    def close(self):
        for sr in (self.sr_own, self.sr_all):
            if sr is not None:
                sr.close()
        self.sr_own = self.sr_all = None


def initial_split(sr_full, pos: torch.Tensor, carry, k: int, min_width: int = 2):
    """Sort a whole particle set with a context for all of it, balance k slabs on the
    per-column work estimate and return (bounds, per-slab lists of arrays [pos, *carry])."""
    sr_full.sort(pos, carry=list(carry))
    n_t = sr_full.stats_geometry()[0]
    toff = sr_full.tile_offsets()
    bounds = slab_bounds(column_weights(toff, n_t), k, min_width if k > 1 else 1)
    col = column_offsets(toff, n_t)
    arrays = [pos, *carry]
    parts = [[a[..., col[bounds[j]]:col[bounds[j + 1]]].contiguous() for a in arrays] for j in range(k)]
    return bounds, parts


class EmulatedSlabs:
    """k slab ranks emulated in one process on one GPU (exchange through LocalFabric):
    the whole set is split once by the balanced column bounds; every ``forces`` call
    then sorts each slab, exchanges emigrants and halos and computes each slab's own
    forces.  ``n_subs`` gives each slab its own subtiles per tile (Section 2.1.3,
    "Subtiles": the decomposition of a domain is its own)."""

    def __init__(self, pos: torch.Tensor, make_context, k: int, n_subs=None, carry=(), min_width: int = 2):
        n = pos.shape[1]
        ids = torch.arange(n, dtype=torch.int64, device=pos.device)
        with make_context(n) as full:
            self.bounds, self.parts = initial_split(full, pos.clone(), [*carry, ids], k, min_width)
            self.n_t = full.stats_geometry()[0]
        self.n = n
        self.exs = [SlabExchange(self.n_t, self.bounds, r, k) for r in range(k)]
        self.ranks = [SlabRank(make_context, ex, n_sub=None if n_subs is None else n_subs[r])
                      for r, ex in enumerate(self.exs)]

    def forces(self, precision: int = 32):
        """One exchange and every slab's forces: per slab (own arrays [pos, *carry, ids],
        accelerations of the own particles, interacting pairs)."""
        outs = [rk.ex.prepare(arr, rk.sort_own(arr)) for rk, arr in zip(self.ranks, self.parts)]
        swapped = LocalFabric.swap_all(self.exs, outs)
        res = []
        for rk, out, (fl, fr) in zip(self.ranks, outs, swapped):
            own, halo = rk.ex.finish(out, fl, fr)
            a, p = rk.forces(own[0], halo, precision)
            res.append((own, a, p))
        self.parts = [r[0] for r in res]
        return res

    def gather(self, res, dtype=None):
        """Accelerations of every particle in the order of the set given at construction,
        and the interacting pairs summed over the slabs."""
        a0 = res[0][1]
        acc = torch.empty((3, self.n), dtype=dtype or a0.dtype, device=a0.device)
        for own, a, _ in res:
            acc[:, own[-1]] = a.to(acc.dtype)
        return acc, sum(r[2] for r in res)

    def close(self):
        for rk in self.ranks:
            rk.close()


def emulated_forces(pos: torch.Tensor, make_context, k: int, precision: int = 32, min_width: int = 2,
                    n_subs=None):
    """Short-range accelerations of all particles computed as k slab ranks emulated in one
    process (one exchange through LocalFabric).  pos: (3, n) float64 on the GPU.  Returns
    (acc in the input order, interacting pairs summed over the ranks, bounds)."""
    em = EmulatedSlabs(pos, make_context, k, n_subs=n_subs, min_width=min_width)
    try:
        acc, pairs = em.gather(em.forces(precision))
    finally:
        em.close()
    return acc, pairs, em.bounds
