"""The seeded input generators: deterministic for a seed, with the shapes,
value ranges and densities their docstrings state (the input recipe)."""
import numpy as np
import pytest

from paper_1809_07444_gb300 import workloads as WL


def test_same_seed_same_inputs_other_seed_other_inputs():
    assert np.array_equal(WL.wator_initial(64, 48, 3), WL.wator_initial(64, 48, 3))
    assert not np.array_equal(WL.wator_initial(64, 48, 3), WL.wator_initial(64, 48, 4))
    assert np.array_equal(WL.traffic_initial(8, 100, 2), WL.traffic_initial(8, 100, 2))
    a, b = WL.sugarscape_initial(64, 64, 5), WL.sugarscape_initial(64, 64, 5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_wator_and_gol_densities():
    k = WL.wator_initial(512, 512, 1)
    assert k.shape == (512, 512) and set(np.unique(k)) <= {0, 1, 2}
    assert abs((k == 1).mean() - 0.30) < 0.01 and abs((k == 2).mean() - 0.03) < 0.005
    g = WL.gol_initial(512, 512, 1)
    assert abs(g.mean() - 0.25) < 0.01


def test_traffic_start():
    v = WL.traffic_initial(256, 1024, 1)
    assert v.shape == (256, 1024) and v.dtype == np.int8
    occ = v >= 0
    assert abs(occ.mean() - 0.2) < 0.01
    assert set(np.unique(v[occ])) == set(range(6)) and (v[~occ] == -1).all()


def test_sugarscape_landscape_and_agents():
    W = H = 200
    cap, a = WL.sugarscape_initial(W, H, 1)
    assert cap.shape == (H, W) and cap.dtype == np.uint8 and cap.max() == 4 and cap.min() == 0
    assert cap[H // 4, W // 4] == 4 and cap[3 * H // 4, 3 * W // 4] == 4  # the two peaks
    assert a.shape[1] == 7 and abs(len(a) / (W * H) - 0.1) < 0.01
    cells = a[:, 1].astype(np.int64) * W + a[:, 0]
    assert len(np.unique(cells)) == len(a)  # one agent per cell
    x, y, sugar, metab, vision, age, max_age = a.T
    assert sugar.min() >= 5 and sugar.max() <= 25 and metab.min() >= 1 and metab.max() <= 4
    assert vision.min() >= 1 and vision.max() <= 6 and max_age.min() >= 60 and max_age.max() <= 100
    assert (age >= 0).all() and (age < max_age).all()


@pytest.mark.parametrize("n", [1, 63, 4097])
def test_nbody_bodies(n):
    rows, seed = WL.nbody_initial(n, 1)
    assert rows.shape == (n, 7)
    assert (rows[:, :3] >= 0).all() and (rows[:, :3] < 1).all() and (rows[:, 3:6] == 0).all()
    assert (rows[:, 6] >= 1e-3).all() and (rows[:, 6] <= 1).all()
    assert np.array_equal(rows.astype(np.float32).astype(np.float64), rows)  # float32-representable


def test_batched_sides_and_served_jobs():
    s = WL.batched_sides(256, 1)
    assert len(s) == 256 and s.min() >= 64 and s.max() <= 1024
    jobs = WL.served_jobs(5000, 2024)
    assert all(len(v) == 5000 for v in jobs.values())
    assert (np.diff(jobs["arrival"]) > 0).all()  # Poisson arrivals, in order
    assert abs(5000 / jobs["arrival"][-1] - 200.0) < 10.0  # at 200 jobs/s
    assert set(np.unique(jobs["app"])) == {0, 1} and abs(jobs["app"].mean() - 0.5) < 0.03
    assert jobs["side"].min() >= 128 and jobs["side"].max() <= 4096
    assert jobs["steps"].min() >= 50 and jobs["steps"].max() <= 1000
