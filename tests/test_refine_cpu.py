"""Host logic of the temporal subtile refinement, with a fake context (no GPU)."""
from types import SimpleNamespace

import pytest

from paper_2112_01508_gb300.refine import SubtileRefiner


class FakeContext:
    """Stands in for ShortRange: force time per pair is a function of n_sub."""

    def __init__(self, cost, n_sub=(1, 1, 1)):
        self.cost = cost
        self.n_sub = n_sub
        self.calls = []  # decomposition of every force call
        self.switches = []
        self.sorted = True

    def set_subtiles(self, ns):
        self.switches.append(tuple(ns))
        self.n_sub = tuple(ns)
        self.sorted = False

    def step(self, refiner):
        refiner.before_sort()
        self.sorted = True  # the sort
        self.calls.append(self.n_sub)
        refiner.after_forces()

    def stats(self):
        return SimpleNamespace(force_kernel_ms=self.cost(self.n_sub[0]) * 1e6, pairs_last=10 ** 6)


def test_trial_every_interval_and_revert_when_slower():
    sr = FakeContext(lambda n: {1: 1.0, 2: 1.3}[n])
    r = SubtileRefiner(sr, interval=16)
    for _ in range(50):
        sr.step(r)
    trials = [i for i, ns in enumerate(sr.calls) if ns != (1, 1, 1)]
    assert trials == [16, 32, 48]
    assert r.current == (1, 1, 1) and r.log.trials == 3 and r.log.kept == 0
    assert sr.switches == [(2, 2, 2), (1, 1, 1)] * 3


def test_refines_while_faster_and_stops_at_the_optimum():
    cost = {1: 3.0, 2: 2.0, 3: 1.5, 4: 1.6, 5: 2.0}
    sr = FakeContext(lambda n: cost[n])
    r = SubtileRefiner(sr, interval=4)
    for _ in range(40):
        sr.step(r)
    assert r.current == (3, 3, 3)
    assert r.log.kept == 2
    assert all(ns in {(3, 3, 3), (4, 4, 4)} for ns in sr.calls[12:])
    kept = [e for e in r.log.events if e[4]]
    assert [e[1] for e in kept] == [(2, 2, 2), (3, 3, 3)]


def test_respects_max_sub():
    sr = FakeContext(lambda n: 1.0 / n, n_sub=(3, 3, 3))
    r = SubtileRefiner(sr, interval=2, max_sub=4)
    for _ in range(20):
        sr.step(r)
    assert r.current == (4, 4, 4)
    assert max(max(ns) for ns in sr.calls) == 4


def test_rejects_bad_interval():
    with pytest.raises(ValueError):
        SubtileRefiner(FakeContext(lambda n: 1.0), interval=1)
