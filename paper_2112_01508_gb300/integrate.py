"""Rung-based leapfrog (Section 2.2.2) over the library's kernels.

Every particle owns a rung l and is kicked every dt / 2^l; positions drift in
2^(n_rung-1) substeps of dt / 2^(n_rung-1) per global step dt.  After each
drift the particles are sorted again into tiles and subtiles (momenta, rungs,
kick states and identifiers carried along), the receivers are the rungs due
at that substep (all particles supply), and p3m_sr_rung_kick applies the kick
with its rung jumps.  The run starts from a synchronised state with the
paper's "fake kick" (forces of all particles, rungs from Eq. rung, half kicks
dt / 2^(l+1)) and ends synchronised.

With a ``LongRange`` context the mesh force kicks every particle whenever
rung 0 is kicked (the paper's rule): dt/2 at the start of a period, dt at the
end of each global step, dt/2 at a synchronisation, after the short-range
kick.  Rungs follow the short-range force alone, as in the paper.
"""
from __future__ import annotations

import torch

from .shortrange import ShortRange


def substep_rung_min(k: int, n_rung: int) -> int:
    """Lowest rung kicked at global substep k >= 1: n_rung - 1 - trailing zeros of k (>= 0)."""
    tz = 0
    while tz < n_rung - 1 and (k >> tz) & 1 == 0:
        tz += 1
    return n_rung - 1 - tz


def rung_leapfrog(sr: ShortRange, pos: torch.Tensor, mom: torch.Tensor, dt: float, eta: float, eps: float,
                  n_steps: int, precision: int = 32, period: int | None = None, carry=(),
                  history: list | None = None, on_substep=None, long_range=None, resort_every: int = 4):
    """Advance (pos, mom) by n_steps global steps of size dt, synchronising after
    every `period` steps (default: once, at the end).

    A period starts synchronised: rungs from Eq. rung on the forces of all
    particles (a fake kick for the first period; the synchronising kick, in
    which every particle is a receiver, for later ones), then half kicks
    dt / 2^(l+1).  pos (3, n) float64 and mom (3, n) float64/float32 are
    reordered in place by the sorts; `carry` lists further per-particle
    tensors to reorder alongside (for example identifiers).  `on_substep(k,
    rung_min)` is called after each substep's kick is enqueued.  The particles
    are sorted again every `resort_every` substeps (1..64, default 4: the paper
    reapplies its memory ordering periodically, and on the 128^3 benchmark set
    every 4th substep is fastest): in between, the library traverses the
    drifted positions with its reach widened by the drift since the sort.
    Returns (rung, kick_state) in the final order.
    """
    if not 1 <= int(resort_every) <= 64:
        raise ValueError("resort_every must be in 1..64")
    n_rung = sr.n_rung
    sub = 2 ** (n_rung - 1)
    period = n_steps if period is None else period
    dev = pos.device
    rung = torch.zeros(sr.n, dtype=torch.int8, device=dev)
    state = torch.zeros(sr.n, dtype=torch.int8, device=dev)
    carried = [mom, rung, state, *carry]
    scratch = [torch.empty_like(t) for t in (pos, *carried)]  # out-of-place sorts, storage swapped back
    sr.sort(pos, carry=carried, scratch=scratch)
    sr.build_pairs()
    acc = sr.forces(pos, precision)
    acc_lr = None if long_range is None else torch.empty((3, sr.n), dtype=long_range.dtype, device=dev)
    half = [dt / 2.0 ** (l + 1) for l in range(n_rung)]
    k = 0
    drifted = False  # the drift of the coming substep was applied with the previous kick
    for step in range(n_steps):
        if step % period == 0:
            sr.assign_rungs(acc, dt, eta, eps, rung)
            state.zero_()
            sr.kick(mom, acc, half, rung, 0)
            if long_range is not None:
                long_range.accel(pos, acc_lr)
                sr.kick(mom, acc_lr, [dt / 2.0])
            k = 0  # substeps since the synchronisation
        last_of_period = (step + 1) % period == 0 or step == n_steps - 1
        for s in range(1, sub + 1):
            k += 1
            if not drifted:
                sr.drift(pos, mom, dt / sub)
            if k % resort_every == 0:
                sr.sort(pos, carry=carried, scratch=scratch)
            lmin = substep_rung_min(k, n_rung)
            sr.build_pairs(None if lmin == 0 else rung, lmin)  # lmin 0: all receivers (each pair once in FP32)
            sr.forces(pos, precision, acc)
            # the kick and the next substep's drift in one pass, unless a synchronisation,
            # a mesh kick or a new period comes between them
            drifted = s < sub or (long_range is None and not last_of_period)
            if drifted:
                sr.rung_kick_drift(mom, acc, rung, state, lmin, k, dt, eta, eps, pos, dt / sub)
            else:
                sr.rung_kick(mom, acc, rung, state, lmin, k, dt, eta, eps, synchronize=last_of_period and s == sub)
            if long_range is not None and s == sub:
                long_range.accel(pos, acc_lr)
                sr.kick(mom, acc_lr, [dt / 2.0 if last_of_period else dt])
            if history is not None:
                history.append(rung.clone())
            if on_substep is not None:
                on_substep(k, lmin)
    return rung, state
