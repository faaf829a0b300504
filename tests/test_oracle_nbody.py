"""Oracle pins for n-body with merging: softened-gravity closed form, superposition, conservation, merge rules."""
import numpy as np
import pytest

import oracle as O
from paper_1809_07444_gb300 import workloads as WL


def _rows(pos, m, vel=None):
    pos = np.asarray(pos, float)
    r = np.zeros((len(pos), 7))
    r[:, 0:3] = pos
    if vel is not None:
        r[:, 3:6] = vel
    r[:, 6] = m
    return r


def test_two_body_step_matches_softened_gravity():
    G, eps, dt = 1.0, 1e-3, 1e-4
    b = O.NBody(_rows([[0.4, 0.5, 0.5], [0.6, 0.5, 0.5]], [0.3, 0.7]), G=G, eps=eps, dt=dt, r_merge=0.0)
    b.step(1)
    d = b.dump()
    # Plummer-softened attraction along the line of centres
    a0 = G * 0.7 * 0.2 / (0.2 ** 2 + eps ** 2) ** 1.5
    a1 = -G * 0.3 * 0.2 / (0.2 ** 2 + eps ** 2) ** 1.5
    assert d[0, 4] == pytest.approx(a0 * dt, rel=1e-13)
    assert d[1, 4] == pytest.approx(a1 * dt, rel=1e-13)
    assert d[0, 1] == pytest.approx(0.4 + a0 * dt * dt, rel=1e-14)
    assert d[0, 5] == 0 and d[0, 6] == 0 and d[0, 2] == 0.5


def test_superposition_of_pair_forces():
    pos = [[0.2, 0.3, 0.4], [0.7, 0.1, 0.5], [0.4, 0.8, 0.9]]
    m = [0.5, 0.25, 0.125]
    full = O.NBody(_rows(pos, m), r_merge=0.0)
    full.step(1)
    v_full = full.dump()[0, 4:7]
    v_sum = np.zeros(3)
    for j in (1, 2):
        pair = O.NBody(_rows([pos[0], pos[j]], [m[0], m[j]]), r_merge=0.0)
        pair.step(1)
        v_sum += pair.dump()[0, 4:7]
    assert np.allclose(v_full, v_sum, rtol=1e-12, atol=0)


def test_symmetric_neighbours_cancel():
    c = np.array([0.5, 0.5, 0.5])
    pos = [c] + [c + 0.1 * np.array(s) for s in np.array(np.meshgrid([-1, 1], [-1, 1], [-1, 1])).T.reshape(-1, 3)]
    b = O.NBody(_rows(pos, [1.0] * 9), r_merge=0.0)
    b.step(1)
    v0 = b.dump()[0, 4:7]
    assert np.abs(v0).max() < 1e-12


def test_momentum_conserved_without_merges():
    rows, _ = WL.nbody_initial(300, 3, margin=0)
    b = O.NBody(rows, r_merge=0.0)
    b.step(20)
    d = b.dump()
    p = (d[:, 7:8] * d[:, 4:7]).sum(0)
    scale = (d[:, 7:8] * np.abs(d[:, 4:7])).sum(0)
    assert np.all(np.abs(p) <= 1e-12 * scale)
    assert len(d) == 300


def test_merges_conserve_mass_and_momentum():
    rng = np.random.default_rng(0)
    n = 400
    pos = 0.5 + 0.05 * rng.random((n, 3))
    vel = rng.normal(0, 1, (n, 3))
    m = rng.uniform(0.1, 1.0, n)
    b = O.NBody(_rows(pos, m, vel), G=1e-4, dt=1e-5, r_merge=4e-3)
    mass0 = m.sum()
    p0 = (m[:, None] * vel).sum(0)
    merges, _ = b.step(5)
    d = b.dump()
    assert len(merges) > 20 and len(d) == n - len(merges)
    assert d[:, 7].sum() == pytest.approx(mass0, rel=1e-13)
    assert np.allclose((d[:, 7:8] * d[:, 4:7]).sum(0), p0, rtol=1e-10, atol=1e-10)
    # the survivor is always the lower id
    assert np.all(merges[:, 1] < merges[:, 2])


def test_merge_chain_only_mutual_partners_merge():
    # ids 0, 1, 2 on a line: p(0)=1, p(1)=0, p(2)=1 -> only (0, 1) merge.
    pos = [[0.5, 0.5, 0.5], [0.5015, 0.5, 0.5], [0.503, 0.5, 0.5]]
    b = O.NBody(_rows(pos, [1.0, 3.0, 1.0]), G=0.0, r_merge=2e-3)
    merges, _ = b.step(1)
    assert merges.tolist() == [[0, 0, 1]]
    d = b.dump()
    assert d[:, 0].tolist() == [0.0, 2.0]
    assert d[0, 1] == pytest.approx((0.5 + 3 * 0.5015) / 4, rel=1e-15)
    assert d[0, 7] == 4.0
    # the merged body now lies 1.875e-3 from body 2: they merge next step
    merges, _ = b.step(1)
    assert merges.tolist() == [[1, 0, 2]]
    assert b.count() == 1


def test_partner_is_lowest_id_within_range():
    # body 2 has both 0 and 1 in range; its partner is 0, so (1, 2) do not merge
    pos = [[0.5, 0.5, 0.5], [0.5033, 0.5, 0.5], [0.5018, 0.5, 0.5]]
    b = O.NBody(_rows(pos, [1.0, 1.0, 1.0]), G=0.0, r_merge=2e-3)
    merges, _ = b.step(1)
    assert merges.tolist() == [[0, 0, 2]]


def test_marginal_pairs_are_counted():
    pos = [[0.5, 0.5, 0.5], [0.5 + 2e-3 + 5e-6, 0.5, 0.5], [0.9, 0.9, 0.9]]
    b = O.NBody(_rows(pos, [1.0] * 3), G=0.0, r_merge=2e-3)
    _, marg = b.step(1, margin=1e-5)
    assert marg == 1


def test_generator_rejects_marginal_pairs():
    rows, used = WL.nbody_initial(4096, 7)
    assert rows.shape == (4096, 7)
    assert np.all(rows.astype(np.float32).astype(np.float64) == rows)
    from scipy.spatial import cKDTree
    pairs = cKDTree(rows[:, :3]).query_pairs(2e-3 + 1e-5, output_type="ndarray")
    if len(pairs):
        d = np.linalg.norm(rows[pairs[:, 0], :3] - rows[pairs[:, 1], :3], axis=1)
        assert not np.any(np.abs(d - 2e-3) < 1e-5)
