"""Parity of the traffic application (Fig. 6g, Nagel-Schreckenberg) with the
oracle: the state hash of both object types after every step, the per-step
event counts (cars entered, left, moved, velocity sum), the sorted object
multisets and the occupancy grid, on open and periodic roads, with ragged
sizes, empty starts and the model's limits; plus the full-size bench
workload every step for 32 steps."""
import numpy as np
import pytest

import oracle as O
from paper_1809_07444_gb300 import workloads as WL
from paper_1809_07444_gb300.apps import Traffic

from helpers import check_invariants

pytestmark = pytest.mark.gpu


def _pair(R, L, v0, seed, **kw):
    return Traffic(R, L, v0, seed, **kw), O.Traffic(R, L, v0, seed, **kw)


def _events(g, before):
    now = g.events()
    return [a - b for a, b in zip(now, before)], now


def _check_state(g, o):
    gc, gs = g.dump()
    oc, os_ = o.dump()
    assert np.array_equal(gc, oc)
    assert np.array_equal(gs, os_)
    occ = np.zeros((g.R, g.L), dtype=np.uint8)
    occ[oc[:, 0], oc[:, 1]] = 1
    assert np.array_equal(g.occupancy(), occ)


@pytest.mark.parametrize("R,L,kw", [
    (37, 211, dict(vmax=5, p=0.25, alpha=0.5)),                      # open roads, ragged sizes
    (16, 500, dict(vmax=5, p=0.25, periodic=True)),                  # ring roads
    (33, 97, dict(vmax=3, p=0.0, alpha=1.0, v_entry=0)),              # deterministic, saturated entry
    (20, 64, dict(vmax=5, p=1.0, alpha=0.3)),                        # always dawdle
    (5, 6, dict(vmax=5, p=0.5, alpha=0.9)),                          # shortest road for vmax 5
])
def test_every_step_matches_the_oracle(R, L, kw):
    v0 = WL.traffic_initial(R, L, 3, density=0.3, vmax=kw["vmax"])
    g, o = _pair(R, L, v0, 17, **kw)
    assert g.hash() == o.hash()
    ev = g.events()
    for s in range(60):
        g.step(1)
        want = o.step(1)[0].tolist()
        got, ev = _events(g, ev)
        assert got == want, s
        assert g.hash() == o.hash(), s
        if s % 20 == 19:
            _check_state(g, o)
    check_invariants(g.heap)
    assert g.heap.stats()["error_flags"] == 0


def test_empty_roads_fill_from_the_sources():
    R, L = 40, 150
    v0 = np.full((R, L), -1, dtype=np.int8)
    g, o = _pair(R, L, v0, 5, vmax=5, p=0.2, alpha=0.7)
    for _ in range(4):
        g.step(25)
        o.step(25)
        assert g.hash() == o.hash()
    _check_state(g, o)
    assert g.count() == o.count() > 0


def test_full_road_ring_is_stuck():
    R, L = 8, 64
    v0 = np.zeros((R, L), dtype=np.int8)  # every cell holds a car at rest
    g, o = _pair(R, L, v0, 5, vmax=5, p=0.3, periodic=True)
    g.step(5)
    o.step(5)
    _check_state(g, o)
    assert (g.dump()[0][:, 2] == 0).all()
    assert g.events()[2] == 0  # nobody moved


def test_bench_workload_every_step():
    # 8192 roads of 4096 cells, 20% occupied (6.7 M cars), open, p 0.25,
    # alpha 0.5: state hash, car count and event counts every step for 32
    # steps, full state at steps 1, 16 and 32
    R, L = 8192, 4096
    v0 = WL.traffic_initial(R, L, 1)
    g, o = _pair(R, L, v0, 1, vmax=5, p=0.25, alpha=0.5)
    prev = g.events()
    for s in range(1, 33):
        g.step(1)
        want = o.step(1)[0].tolist()
        now = g.events()
        assert [a - b for a, b in zip(now, prev)] == want, s
        prev = now
        assert g.hash() == o.hash(), s
        assert g.count() == o.count(), s
        if s in (1, 16, 32):
            _check_state(g, o)
    assert g.heap.stats()["error_flags"] == 0
    check_invariants(g.heap)
