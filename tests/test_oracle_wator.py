"""Oracle pins for wa-tor: closed forms on hand-built grids, conservation laws and movement locality."""
import numpy as np
import pytest

import oracle as O
from paper_1809_07444_gb300 import workloads as WL

E, F, S = WL.EMPTY, WL.FISH, WL.SHARK


def _nbrs(x, y, W, H):
    return [(x, (y - 1) % H), ((x + 1) % W, y), (x, (y + 1) % H), ((x - 1) % W, y)]  # N E S W


def test_lone_shark_starves_after_energy0_steps():
    k = np.zeros((8, 8), np.uint8)
    k[3, 3] = S
    w = O.Wator(8, 8, k, seed=1)
    for t in range(4):
        ev = w.step(1)
        assert w.counts() == (0, 1)
        assert ev[0, 3] == 0
        _, sh = w.dump()
        assert sh[0, 3] == 5 - (t + 1) and sh[0, 2] == t + 1  # energy, timer
    ev = w.step(1)
    assert w.counts() == (0, 0) and ev[0, 3] == 1


def test_lone_fish_moves_to_drawn_neighbour_and_breeds_at_three():
    W = H = 16
    k = np.zeros((H, W), np.uint8)
    x, y = 5, 7
    k[y, x] = F
    w = O.Wator(W, H, k, seed=42)
    for t in range(3):
        c = y * W + x
        x, y = _nbrs(x, y, W, H)[O.rand(42, 0, t, c) % 4]
        w.step(1)
        f, _ = w.dump()
        if t < 2:
            assert f.tolist() == [[x, y, t + 1]]
    # third move: timer reached 3, a newborn stays in the cell left behind
    assert len(f) == 2
    assert [x, y, 0] in f.tolist()


def test_contended_cell_goes_to_lowest_mover_index():
    # 3x3 torus full of fish except the centre: its four neighbours all have
    # the centre as their only empty neighbour; the fish in cell 1 (x=1, y=0)
    # has the lowest index and wins.
    k = np.full((3, 3), F, np.uint8)
    k[1, 1] = E
    w = O.Wator(3, 3, k, seed=3)
    w.step(1)
    g = w.grid()
    want = np.full((3, 3), F, np.uint8)
    want[0, 1] = E
    assert np.array_equal(g, want)
    f, _ = w.dump()
    assert all(row[2] == 1 for row in f)  # every fish aged one step, none bred


def test_shark_prefers_fish_and_gains_energy():
    k = np.full((4, 4), F, np.uint8)
    k[0, 0] = S
    w = O.Wator(4, 4, k, seed=11)
    ev = w.step(1)
    assert ev[0].tolist() == [0, 1, 0, 0, 0, 1]  # no fish can move; the shark moves once
    assert w.counts() == (14, 1)
    _, sh = w.dump()
    assert sh[0, 3] == 5 - 1 + 3 and sh[0, 2] == 1
    tx, ty = _nbrs(0, 0, 4, 4)[O.rand(11, 1, 0, 0) % 4]
    assert (sh[0, 0], sh[0, 1]) == (tx, ty)
    assert w.grid()[0, 0] == E


def test_shark_breeds_on_tenth_step_among_plenty_of_fish():
    k = np.full((32, 32), F, np.uint8)
    k[10, 10] = S
    w = O.Wator(32, 32, k, seed=5)
    for t in range(9):
        ev = w.step(1)
        assert ev[0, 1] == 1 and w.counts()[1] == 1
    ev = w.step(1)
    assert ev[0, 1] == 1 and ev[0, 2] == 1
    _, sh = w.dump()
    assert sorted((r[2], r[3]) for r in sh) == [(0, 5), (0, 5 + 10 * 2)]


def test_lone_fish_moves_every_step_and_breeds_on_the_third():
    k = np.zeros((5, 5), np.uint8)
    k[2, 2] = F
    w = O.Wator(5, 5, k, seed=3)
    ev = w.step(3)
    assert ev[:, 4].tolist() == [1, 1, 1] and ev[:, 0].tolist() == [0, 0, 1]
    assert w.counts() == (2, 0)


def test_fish_only_full_grid_never_moves():
    k = np.full((5, 5), F, np.uint8)
    w = O.Wator(5, 5, k, seed=1)
    ev = w.step(7)
    assert ev.sum() == 0
    f, _ = w.dump()
    assert len(f) == 25 and all(r[2] == 7 for r in f)


@pytest.mark.parametrize("W,H,seed,steps", [(64, 64, 1, 60), (17, 9, 2, 80)])
def test_conservation_exclusivity_and_locality(W, H, seed, steps):
    k0 = WL.wator_initial(W, H, seed)
    w = O.Wator(W, H, k0, seed=seed)
    nf, ns = w.counts()
    assert nf == (k0 == F).sum() and ns == (k0 == S).sum()
    prev = w.grid().copy()
    for t in range(steps):
        ev = w.step(1)[0]
        f2, s2 = w.counts()
        assert f2 == nf + ev[0] - ev[1]
        assert s2 == ns + ev[2] - ev[3]
        # births happen only on a move; a shark eats only by moving; nobody moves twice
        assert ev[0] <= ev[4] <= nf and ev[2] <= ev[5] and ev[1] <= ev[5] <= ns - ev[3]
        nf, ns = f2, s2
        g = w.grid()
        f, s = w.dump()
        # one agent per cell and the grid agrees with the objects
        occ = np.zeros((H, W), np.uint8)
        for x, y, *_ in f:
            assert occ[y, x] == 0
            occ[y, x] = F
        for x, y, *_ in s:
            assert occ[y, x] == 0
            occ[y, x] = S
        assert np.array_equal(occ, g)
        assert (s[:, 3] >= 1).all() if len(s) else True
        # every agent is where an agent of its kind was, or next to such a cell
        for kind, objs in ((F, f), (S, s)):
            for x, y, *_ in objs:
                near = [(x, y)] + _nbrs(x, y, W, H)
                assert any(prev[yy, xx] == kind for xx, yy in near)
        prev = g.copy()


def test_seed_changes_trajectory_and_hash_is_state_function():
    k0 = WL.wator_initial(32, 32, 4)
    a, b, c = O.Wator(32, 32, k0, seed=4), O.Wator(32, 32, k0, seed=4), O.Wator(32, 32, k0, seed=5)
    a.step(10)
    b.step(10)
    c.step(10)
    assert a.hash() == b.hash()
    assert a.hash() != c.hash()
