"""Slab decomposition of the periodic box for the short-range force, emulated on
one GPU (the paper's domains, Section 2.1.2 "Parallelisation", and its
tile-level pairing of neighbouring domains, Section 2.1.3 "Tiles").

The box is cut along x into K slabs of whole tile columns.  Tiles are at least
x_r wide, so the receivers of a slab need as suppliers only the particles of one
tile column on each side of it (the halo).  Slab boundaries follow the prefix of
a per-column work estimate, the sum over the column's tiles of (particles per
tile)^2 -- a tile's pair count up to a constant -- which addresses the load
imbalance under clustering that the paper names as its scheme's main weakness.

Every run of this library has one GPU, so the domains are emulated: each is
computed by its own ShortRange context on its particles plus its halo, with
only its own particles as receivers.  The accelerations equal the whole-box
ones (the same pairs, summed in another order).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from .shortrange import ShortRange


@dataclass
class Domain:
    tiles: tuple[int, int]   # tile columns [t0, t1) along x
    local: np.ndarray        # indices of the particles in the slab
    halo: np.ndarray         # indices of the particles in the columns t0 - 1 and t1 (periodic)


def tile_indices(pos: np.ndarray, n_t: int, box: float = 1.0) -> np.ndarray:
    """(3, n) integer tile coordinates floor(x n_t / L), clipped to n_t - 1."""
    t = np.floor(np.asarray(pos, dtype=np.float64) * (n_t / box)).astype(np.int64)
    return np.clip(t, 0, n_t - 1)


def column_weights(tiles: np.ndarray, n_t: int) -> np.ndarray:
    """Work estimate per tile column along x: sum over its tiles of count^2."""
    flat = (tiles[0] * n_t + tiles[1]) * n_t + tiles[2]
    counts = np.bincount(flat, minlength=n_t ** 3).astype(np.float64).reshape(n_t, n_t, n_t)
    return (counts ** 2).sum(axis=(1, 2))


def slab_bounds(weights: np.ndarray, k: int) -> list[int]:
    """Boundaries 0 = b_0 < ... < b_k = n_t of k slabs of whole columns: each slab in
    turn takes the prefix closest to an equal share of the weight still to assign
    (a heavy column then sits in a slab of its own and the rest is spread over the
    others); every slab keeps at least one column."""
    n_t = len(weights)
    if not 1 <= k <= n_t:
        raise ValueError("need 1 <= k <= number of tile columns")
    c = np.concatenate([[0.0], np.cumsum(weights, dtype=np.float64)])
    b = [0]
    for j in range(1, k):
        start = b[-1]
        target = c[start] + (c[-1] - c[start]) / (k - j + 1)
        lo, hi = start + 1, n_t - (k - j)  # leave one column for each slab still to come
        t = min(max(int(np.searchsorted(c, target, side="left")), lo), hi)
        if t - 1 >= lo and abs(c[t - 1] - target) <= abs(c[t] - target):
            t -= 1
        b.append(t)
    b.append(n_t)
    return b


def decompose(pos: np.ndarray, n_t: int, k: int, box: float = 1.0, balance: bool = True) -> list[Domain]:
    """Split the particles into k slabs with their one-column halos."""
    tiles = tile_indices(pos, n_t, box)
    w = column_weights(tiles, n_t) if balance else np.ones(n_t)
    b = slab_bounds(w, k)
    tx = tiles[0]
    out = []
    for j in range(k):
        t0, t1 = b[j], b[j + 1]
        local = np.flatnonzero((tx >= t0) & (tx < t1))
        if k == 1:
            halo = np.zeros(0, dtype=np.int64)
        else:
            left, right = (t0 - 1) % n_t, t1 % n_t
            halo = np.flatnonzero(((tx == left) | (tx == right)) & ~((tx >= t0) & (tx < t1)))
        out.append(Domain((t0, t1), local, halo))
    return out


def emulated_forces(pos: torch.Tensor, x_s: float, x_r: float, G_m: float, k: int, softening: str = "bspline",
                    eps: float = 0.0, n_sub=2, precision: int = 32, box: float = 1.0, balance: bool = True):
    """Short-range accelerations of all particles computed as k slab domains, one
    context per domain.  pos: (3, n) float64 on the GPU, any order.  Returns
    (acc in the input order, interacting pairs summed over the domains, domains)."""
    n = pos.shape[1]
    n_t = int(np.floor(box / x_r))
    doms = decompose(pos.cpu().numpy(), n_t, k, box, balance)
    dt = torch.float32 if precision == 32 else torch.float64
    acc = torch.empty((3, n), dtype=dt, device=pos.device)
    pairs = 0
    for d in doms:
        idx = np.concatenate([d.local, d.halo])
        m = len(idx)
        if len(d.local) == 0:
            continue
        sub = pos[:, torch.from_numpy(idx).to(pos.device)].contiguous()
        own = torch.zeros(m, dtype=torch.int8, device=pos.device)
        own[:len(d.local)] = 1                 # receivers: the slab's own particles
        ids = torch.arange(m, dtype=torch.int32, device=pos.device)
        with ShortRange(m, x_s, x_r, G_m, softening=softening, eps=eps, n_sub=n_sub, box=box,
                        device=pos.device) as sr:
            sr.sort(sub, carry=[own, ids])
            sr.build_pairs(own, 1)
            a = sr.forces(sub, precision)
            pairs += sr.stats().pairs_last
        sel = own.bool()
        gidx = torch.from_numpy(idx).to(pos.device)[ids[sel].long()]
        acc[:, gidx] = a[:, sel]
    return acc, pairs, doms
