"""Pins of the sugarscape oracle (Fig. 6f; Epstein and Axtell's rules M,
G_alpha and R): closed forms of lone agents and single cells, the movement
rule's order of preference, the claim rule, and invariants of random runs.
"""
import numpy as np
import pytest

import oracle as O

W = H = 17


def _one(x, y, sugar, metab, vision, age=0, max_age=1000):
    return np.array([[x, y, sugar, metab, vision, age, max_age]], dtype=np.int32)


def test_lone_agent_takes_the_best_cell_in_sight_then_lives_on_growback():
    cap = np.zeros((H, W), np.uint8)
    cap[8, 11] = 4  # 3 cells east of the agent
    cap[8, 2] = 4   # 6 cells west: out of sight (vision 4)
    s = O.Sugarscape(W, H, cap, _one(8, 8, 10, 2, 4), 1)
    sugar = 10
    for t in range(12):
        ev = s.step(1)[0]
        a, sg = s.dump()
        gain = 4 if t == 0 else 1  # the cell regrows by 1 a step after each harvest
        sugar += gain - 2
        assert a[:, :2].tolist() == [[11, 8]]
        assert a[0, 2] == sugar and a[0, 5] == t + 1
        assert ev.tolist() == [1 if t == 0 else 0, 0, 0, 0, gain]
        assert sg[8, 11] == 1 and sg[8, 2] == 4


@pytest.mark.parametrize("alpha,cap_v", [(1, 4), (2, 4), (1, 3), (3, 2)])
def test_growback_after_a_harvest(alpha, cap_v):
    cap = np.zeros((H, W), np.uint8)
    cap[3, 3] = cap_v
    s = O.Sugarscape(W, H, cap, _one(3, 3, 50, 1, 1), 1, alpha=alpha)
    s.step(1)
    # the agent harvests its cell every step: the cell shows min(alpha, cap)
    for _ in range(5):
        assert s.dump()[1][3, 3] == min(alpha, cap_v)
        s.step(1)


def test_untouched_landscape_stays_at_capacity():
    rng = np.random.default_rng(1)
    cap = rng.integers(0, 5, (H, W)).astype(np.uint8)
    s = O.Sugarscape(W, H, cap, np.zeros((0, 7), np.int32), 1)
    s.step(10)
    assert np.array_equal(s.dump()[1], cap.astype(np.int32))
    assert s.count() == 0


@pytest.mark.parametrize("s0,m", [(0, 1), (5, 2), (7, 1), (12, 4)])
def test_starvation_step_and_replacement(s0, m):
    cap = np.zeros((H, W), np.uint8)
    s = O.Sugarscape(W, H, cap, _one(4, 4, s0, m, 1), 3)
    death = s0 // m  # after k + 1 steps the sugar is s0 - (k + 1) m, below 0 first at k = s0 // m
    for t in range(death + 1):
        ev = s.step(1)[0]
        a, _ = s.dump()
        assert len(a) == 1  # the population is constant
        if t < death:
            assert ev[1] == 0 and a[0, 2] == s0 - (t + 1) * m
        else:
            assert ev[1] == 1
            assert a[0, 5] == 0  # the replacement is newborn
            assert 5 <= a[0, 2] <= 25 and 1 <= a[0, 3] <= 4 and 1 <= a[0, 4] <= 6 and 60 <= a[0, 6] <= 100


def test_death_at_maximum_age():
    cap = np.full((H, W), 4, np.uint8)
    s = O.Sugarscape(W, H, cap, _one(4, 4, 100, 1, 1, age=0, max_age=7), 3)
    ev = s.step(7)
    assert ev[:6, 2].sum() == 0 and ev[6, 2] == 1 and ev[:, 1].sum() == 0


def test_more_sugar_beats_nearer_and_nearer_beats_farther():
    cap = np.zeros((H, W), np.uint8)
    cap[8, 10] = 3  # east, distance 2
    cap[5, 8] = 3   # north, distance 3: same sugar, farther
    cap[8, 4] = 4   # west, distance 4: more sugar
    s = O.Sugarscape(W, H, cap, _one(8, 8, 10, 1, 4), 1)
    s.step(1)
    assert s.dump()[0][0, :2].tolist() == [4, 8]
    cap[8, 4] = 0
    s = O.Sugarscape(W, H, cap, _one(8, 8, 10, 1, 4), 1)
    s.step(1)
    assert s.dump()[0][0, :2].tolist() == [10, 8]


def test_contested_cell_goes_to_the_lowest_cell_index():
    cap = np.zeros((H, W), np.uint8)
    cap[8, 8] = 4
    agents = np.array([[8, 6, 10, 1, 2, 0, 1000],    # cell 6 * 17 + 8 = 110, two north of the target
                       [10, 8, 10, 1, 2, 0, 1000]],  # cell 8 * 17 + 10 = 146, two east of it
                      dtype=np.int32)
    s = O.Sugarscape(W, H, cap, agents, 1)
    ev = s.step(1)[0]
    a, _ = s.dump()
    assert ev[0] == 1
    assert sorted(a[:, :2].tolist()) == [[8, 8], [10, 8]]  # the northern agent moved, the other stayed


def test_invariants_of_random_runs():
    rng = np.random.default_rng(4)
    Wb, Hb = 40, 30
    cap = rng.integers(0, 5, (Hb, Wb)).astype(np.uint8)
    cells = rng.choice(Wb * Hb, 300, replace=False)
    agents = np.stack([cells % Wb, cells // Wb, rng.integers(5, 26, 300), rng.integers(1, 5, 300),
                       rng.integers(1, 7, 300), np.zeros(300, int), rng.integers(60, 101, 300)], 1).astype(np.int32)
    s = O.Sugarscape(Wb, Hb, cap, agents, 9)
    for t in range(120):
        ev = s.step(1)[0]
        a, sg = s.dump()
        assert len(a) == 300
        assert len({(x, y) for x, y in a[:, :2].tolist()}) == 300  # one agent per cell
        assert ((sg >= 0) & (sg <= cap)).all()
        assert ((a[:, 2] >= 0) & (a[:, 7] == 0)).all()  # no live agent below zero sugar or dead
        assert (a[:, 5] == 0).sum() == ev[1] + ev[2]  # one newborn per death
        assert ev[3] <= ev[1] + ev[2]
