"""Pins of the traffic oracle (Fig. 6g, the Nagel-Schreckenberg model):
closed forms of the model's limits and its exactly known flows.

- one car on an empty open road with no randomisation accelerates by one
  cell per step up to vmax and leaves when it passes the end;
- a car that always dawdles: from rest it never moves, from vmax it settles
  at vmax - 1;
- the deterministic model (p = 0) on a ring carries the flow
  J = min(rho * vmax, 1 - rho) (the fundamental diagram of the deterministic
  NaSch model);
- with vmax = 1 the parallel-update model on a ring is exactly solvable:
  J = (1 - sqrt(1 - 4 (1 - p) rho (1 - rho))) / 2 (Schadschneider and
  Schreckenberg, J. Phys. A 26, L679, 1993);
- with vmax = 1, p = 0 and an entry probability of 1 the left boundary
  admits a car every second step;
- invariants on random open roads: one car per cell, 0 <= v <= vmax, cars
  conserved up to entries and exits, each source enters or is blocked at
  most once per step.
"""
import numpy as np
import pytest

import oracle as O


def _empty(R, L):
    return np.full((R, L), -1, dtype=np.int8)


@pytest.mark.parametrize("vmax,L", [(5, 100), (3, 50), (1, 10), (7, 333)])
def test_single_car_accelerates_then_leaves(vmax, L):
    v0 = _empty(1, L)
    v0[0, 0] = 0
    t = O.Traffic(1, L, v0, 1, vmax=vmax, p=0.0, alpha=0.0)
    x = 0
    for s in range(10 * L):
        v = min(s + 1, vmax)
        x += v
        ev = t.step(1)[0]
        cars, _ = t.dump()
        if x >= L:
            assert len(cars) == 0 and ev[1] == 1  # left at the step it passed the end
            break
        assert cars.tolist() == [[0, x, v]], s
        assert ev.tolist() == [0, 0, 1, v]
    else:
        pytest.fail("the car never left")
    assert t.step(3)[:, :2].sum() == 0


@pytest.mark.parametrize("v_start", [0, 5])
def test_car_that_always_dawdles(v_start):
    v0 = _empty(1, 1000)
    v0[0, 0] = v_start
    t = O.Traffic(1, 1000, v0, 1, vmax=5, p=1.0, alpha=0.0)
    for s in range(50):
        t.step(1)
        cars, _ = t.dump()
        if v_start == 0:
            assert cars.tolist() == [[0, 0, 0]]
        else:
            assert cars.tolist() == [[0, 4 * (s + 1), 4]]


def _ring_flow(R, L, rho, vmax, p, seed, warm, meas):
    rng = np.random.default_rng(seed)
    v0 = _empty(R, L)
    for r in range(R):
        v0[r, rng.choice(L, int(rho * L), replace=False)] = 0
    t = O.Traffic(R, L, v0, seed, vmax=vmax, p=p, periodic=True)
    n0 = t.count()
    t.step(warm)
    ev = t.step(meas)
    assert t.count() == n0 and ev[:, :2].sum() == 0  # a ring neither gains nor loses cars
    return ev[:, 3].sum() / (R * L * meas)


@pytest.mark.parametrize("rho", [0.1, 0.15, 0.2, 0.7])
def test_deterministic_ring_flow(rho):
    assert abs(_ring_flow(8, 1000, rho, 5, 0.0, 3, 1500, 500) - min(rho * 5, 1 - rho)) < 1e-9


@pytest.mark.parametrize("rho", [0.3, 0.7])
def test_vmax1_ring_flow_matches_the_exact_solution(rho):
    q = 0.75
    exact = (1 - np.sqrt(1 - 4 * q * rho * (1 - rho))) / 2
    assert abs(_ring_flow(64, 1000, rho, 1, 0.25, 4, 300, 300) - exact) < 0.003


def test_saturated_entry_admits_a_car_every_second_step():
    t = O.Traffic(1, 200, _empty(1, 200), 1, vmax=1, p=0.0, alpha=1.0, v_entry=1)
    ev = t.step(400)
    assert ev[0, 0] == 1 and (ev[1:399, 0].reshape(-1, 2).sum(1) == 1).all()
    assert ev[300:, 0].mean() == 0.5 and ev[300:, 1].mean() == 0.5  # in = out = 1/2


def test_invariants_on_random_open_roads():
    rng = np.random.default_rng(5)
    R, L, vmax = 16, 300, 5
    v0 = np.where(rng.random((R, L)) < 0.25, rng.integers(0, vmax + 1, (R, L)), -1).astype(np.int8)
    t = O.Traffic(R, L, v0, 9, vmax=vmax, p=0.3, alpha=0.6)
    n = t.count()
    entered = 0
    for s in range(200):
        ev = t.step(1)[0]
        cars, src = t.dump()
        assert len(cars) == n + ev[0] - ev[1]
        n = len(cars)
        assert len({(r, x) for r, x, _ in cars.tolist()}) == n  # one car per cell
        assert ((cars[:, 2] >= 0) & (cars[:, 2] <= vmax)).all()
        assert ((cars[:, 1] >= 0) & (cars[:, 1] < L)).all()
        entered += ev[0]
        assert src[:, 1].sum() == entered
        assert (src[:, 1] + src[:, 2] <= s + 1).all()
        assert ev[2] <= n - ev[0] + ev[1] and ev[3] <= vmax * ev[2]


@pytest.mark.parametrize("p", [0.0, 0.25, 0.5, 1.0 / 3.0, 0.999999, 1.0])
def test_probability_thresholds_agree_with_the_binding(p):
    # both sides turn a probability into the 32-bit threshold on their own;
    # the GPU path's draws are compared against the binding's value
    pytest.importorskip("torch")
    from paper_1809_07444_gb300.apps import prob_threshold

    assert O.prob_threshold(p) == prob_threshold(p)
    assert O.prob_threshold(p) == int(p * 2 ** 32) if p < 1 else O.prob_threshold(p) == 2 ** 32
