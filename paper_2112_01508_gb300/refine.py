"""Subtile refinement, temporal and per region (Section 2.1.3, "Subtiles";
Section 4, subtile refinement figure).

The paper lets each process check, every 16th time step, whether one more
subdivision of its tiles pays: it applies the refined subtiling for one
short-range computation, compares the measured time with its record for the
current subtiling, and keeps the refinement only if it was faster.  Each
process decides for its own domain, so the decomposition adapts in space as
well as in time.  ``SubtileRefiner`` applies the rule to one context (one
decomposition for the whole box); ``RegionRefiner`` applies it to every slab
of a slab decomposition (``slabs.SlabRank``: a rank's domain, or a region of one
GPU's box emulated as one), each slab keeping its own subtiling.  The tiles are
cubes, so all three dimensions are refined in lockstep (the "as cubic as
possible" rule).

Because the receivers change from substep to substep under the rung scheme,
the record and the trial are compared as device time per interacting pair
(the pair count does not depend on the subtiling).
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass
class RefinementLog:
    trials: int = 0
    kept: int = 0
    events: list = field(default_factory=list)  # (force call index, trial n_sub, record, trial time, kept)


class SubtileRefiner:
    """Drive ShortRange.set_subtiles around the force calls of a step loop.

    Call ``before_sort()`` before each step's sort and ``after_forces()`` after
    its force call.  Every ``interval`` force calls the refiner reads the
    force-kernel time of the current subtiling (the call before a trial) and
    runs the next call with one more subtile per dimension; the trial's
    decomposition is kept if its time per pair is lower, otherwise the previous
    one returns at the next sort.  Reading a time synchronises the stream, so
    this happens only twice per interval.
    """

    def __init__(self, sr, interval: int = 16, max_sub: int = 8):
        if interval < 2:
            raise ValueError("interval must be >= 2")
        self.sr = sr
        self.interval = int(interval)
        self.max_sub = int(max_sub)
        self.current = tuple(sr.n_sub)
        self.calls = 0
        self.record = None
        self.trial = None
        self.log = RefinementLog()

    def before_sort(self):
        c = self.calls
        if c > 0 and c % self.interval == 0 and self.record is not None and max(self.current) < self.max_sub:
            self.trial = tuple(v + 1 for v in self.current)
            self.sr.set_subtiles(self.trial)
        elif tuple(self.sr.n_sub) != self.current:
            self.sr.set_subtiles(self.current)  # a rejected trial: back to the kept decomposition

    def after_forces(self):
        c = self.calls
        self.calls += 1
        if self.trial is not None:
            t = self._time_per_pair()
            kept = t < self.record
            self.log.trials += 1
            self.log.events.append((c, self.trial, self.record, t, kept))
            if kept:
                self.log.kept += 1
                self.current = self.trial
                self.record = t
            self.trial = None
        elif (c + 1) % self.interval == 0:
            self.record = self._time_per_pair()

    def _time_per_pair(self) -> float:
        st = self.sr.stats()
        return st.force_kernel_ms / max(st.pairs_last, 1)


class RegionRefiner:
    """Per-region subtile refinement: one ``SubtileRefiner`` per slab (anything with
    ``n_sub``, ``set_subtiles`` and ``stats``, such as ``slabs.SlabRank``), each deciding
    from the kernel time per pair of its own slab.  Call ``before_sort()`` before the
    slabs' force contexts sort and ``after_forces()`` after every slab's force call."""

    def __init__(self, slabs, interval: int = 16, max_sub: int = 8):
        self.refiners = [SubtileRefiner(s, interval, max_sub) for s in slabs]

    def before_sort(self):
        for r in self.refiners:
            r.before_sort()

    def after_forces(self):
        for r in self.refiners:
            r.after_forces()

    @property
    def current(self) -> list:
        return [r.current for r in self.refiners]

    @property
    def logs(self) -> list:
        return [r.log for r in self.refiners]
