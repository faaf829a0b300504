"""Oracle pins for game of life: closed forms (blinker, block, glider) and the textbook B3/S23 rule."""
import numpy as np
import pytest

import oracle as O
from paper_1809_07444_gb300 import workloads as WL


def _grid(W, H, cells):
    g = np.zeros((H, W), dtype=np.uint8)
    for x, y in cells:
        g[y % H, x % W] = 1
    return g


def _textbook_life(g):
    """B3/S23 on a torus with the Moore neighbourhood, via shifted copies."""
    n = sum(np.roll(np.roll(g, dy, 0), dx, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy) != (0, 0))
    return ((n == 3) | ((g == 1) & (n == 2))).astype(np.uint8), n


def test_empty_grid_stays_empty():
    g = O.Gol(16, 16, np.zeros((16, 16), np.uint8))
    g.step(10)
    assert g.alive_count() == 0


def test_blinker_has_period_two():
    start = _grid(8, 8, [(2, 3), (3, 3), (4, 3)])
    g = O.Gol(8, 8, start)
    g.step(1)
    assert np.array_equal(g.grid(), _grid(8, 8, [(3, 2), (3, 3), (3, 4)]))
    g.step(1)
    assert np.array_equal(g.grid(), start)
    cells, alive = g.dump()
    # counts are those of the vertical phase: the centre sees 2 neighbours,
    # the cells that were born at the ends saw 3
    assert cells[3 * 8 + 3, 1] == 2 and cells[3 * 8 + 2, 1] == 3 and cells[3 * 8 + 4, 1] == 3
    assert sorted(map(tuple, alive)) == [(2, 3), (3, 3), (4, 3)]


def test_block_is_still_life():
    start = _grid(10, 10, [(4, 4), (5, 4), (4, 5), (5, 5)])
    g = O.Gol(10, 10, start)
    for _ in range(5):
        g.step(1)
        assert np.array_equal(g.grid(), start)
    cells, _ = g.dump()
    assert all(cells[y * 10 + x, 1] == 3 for x, y in [(4, 4), (5, 4), (4, 5), (5, 5)])


def test_glider_translates_diagonally_and_wraps():
    # glider heading +x, +y: after 4 generations the same shape moved by (1, 1)
    shape = [(1, 0), (2, 1), (0, 2), (1, 2), (2, 2)]
    W = H = 64
    g = O.Gol(W, H, _grid(W, H, shape))
    g.step(4)
    assert np.array_equal(g.grid(), _grid(W, H, [(x + 1, y + 1) for x, y in shape]))
    g.step(4 * 64 - 4)  # full wrap around the 64-torus
    assert np.array_equal(g.grid(), _grid(W, H, shape))
    assert g.alive_count() == 5


@pytest.mark.parametrize("W,H,seed,gens", [(64, 64, 1, 100), (13, 7, 2, 40), (3, 3, 3, 10)])
def test_matches_textbook_rule(W, H, seed, gens):
    start = WL.gol_initial(W, H, seed)
    g = O.Gol(W, H, start)
    ref = start.copy()
    for _ in range(gens):
        g.step(1)
        ref, n = _textbook_life(ref)
        cells, alive = g.dump()
        assert np.array_equal(cells[:, 0].reshape(H, W), ref)
        assert np.array_equal(cells[:, 1].reshape(H, W), n)
        assert np.array_equal(cells[:, 2], np.arange(W * H))
        ys, xs = np.nonzero(ref)
        want = np.array(sorted(zip(xs, ys)), dtype=np.int32).reshape(-1, 2)
        assert np.array_equal(alive, want)


def test_hash_tracks_state():
    start = WL.gol_initial(32, 32, 9)
    a, b = O.Gol(32, 32, start), O.Gol(32, 32, start)
    a.step(5)
    b.step(5)
    assert a.hash() == b.hash()
    b.step(1)
    assert a.hash() != b.hash()
