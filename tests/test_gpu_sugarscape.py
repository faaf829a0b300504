"""Parity of the sugarscape application (Fig. 6f; Epstein-Axtell rules M,
G_alpha, R) with the oracle: the agents' state hash and the events every
step, the sorted agents and the sugar of every cell at sampled steps, on
ragged and minimum-size grids, sparse, dense and empty starts, two growback
rates, and the full-size bench workload every step for 30 steps."""
import numpy as np
import pytest

import oracle as O
from paper_1809_07444_gb300 import workloads as WL
from paper_1809_07444_gb300.apps import Sugarscape

from helpers import check_invariants

pytestmark = pytest.mark.gpu


def _pair(W, H, cap, agents, seed, **kw):
    return Sugarscape(W, H, cap, agents, seed, **kw), O.Sugarscape(W, H, cap, agents, seed, **kw)


def _check(g, o):
    ga, gs = g.dump()
    oa, os_ = o.dump()
    assert np.array_equal(ga, oa)
    assert np.array_equal(gs, os_)


@pytest.mark.parametrize("W,H,density,kw", [
    (64, 64, 0.1, {}),                 # the bench recipe, small
    (37, 29, 0.3, dict(alpha=2)),      # ragged, faster growback
    (13, 13, 0.5, {}),                 # the smallest torus for vision 6
    (50, 40, 0.9, dict(max_age=(5, 12))),  # crowded, many deaths by age
])
def test_every_step_matches_the_oracle(W, H, density, kw):
    cap, agents = WL.sugarscape_initial(W, H, 3, density)
    if "max_age" in kw:
        agents[:, 6] = np.clip(agents[:, 6], *kw["max_age"])
        agents[:, 5] = np.minimum(agents[:, 5], agents[:, 6] - 1)
    g, o = _pair(W, H, cap, agents, 21, **kw)
    assert g.hash() == o.hash()
    prev = g.events()
    for s in range(80):
        g.step(1)
        want = o.step(1)[0].tolist()
        now = g.events()
        assert [a - b for a, b in zip(now, prev)] == want, s
        prev = now
        assert g.hash() == o.hash(), s
        if s % 20 == 19:
            _check(g, o)
    check_invariants(g.heap)
    assert g.heap.stats()["error_flags"] == 0


def test_landscape_without_agents_stays_full():
    cap, _ = WL.sugarscape_initial(40, 40, 2)
    g, o = _pair(40, 40, cap, np.zeros((0, 7), np.int32), 5)
    g.step(5)
    o.step(5)
    _check(g, o)
    assert np.array_equal(g.dump()[1], cap.astype(np.int32))


def test_bench_workload_every_step():
    # 4096 x 4096, 10% of the cells hold an agent (1.68 M agents): agents'
    # state hash and event counts every step for 30 steps, sorted agents and
    # the sugar of every cell at steps 1, 15 and 30
    W = H = 4096
    cap, agents = WL.sugarscape_initial(W, H, 1)
    g, o = _pair(W, H, cap, agents, 1)
    prev = g.events()
    for s in range(1, 31):
        g.step(1)
        want = o.step(1)[0].tolist()
        now = g.events()
        assert [a - b for a, b in zip(now, prev)] == want, s
        prev = now
        assert g.hash() == o.hash(), s
        if s in (1, 15, 30):
            _check(g, o)
    assert g.count() == o.count() == len(agents)
    assert g.heap.stats()["error_flags"] == 0
    check_invariants(g.heap)
