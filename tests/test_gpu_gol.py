"""GPU parity of game of life with the oracle (bit-exact Cell and Alive multisets every generation)."""
import numpy as np
import pytest

import oracle as O
from paper_1809_07444_gb300 import workloads as WL
from paper_1809_07444_gb300.apps import Gol

from helpers import check_invariants

pytestmark = pytest.mark.gpu


def _run_pair(W, H, start, gens, full_every=1):
    gpu, ref = Gol(W, H, start), O.Gol(W, H, start)
    assert gpu.hash() == ref.hash()
    for g in range(1, gens + 1):
        gpu.step(1)
        ref.step(1)
        assert gpu.hash() == ref.hash(), "generation %d" % g
        if g % full_every == 0 or g == gens:
            cg, ag = gpu.dump()
            cr, ar = ref.dump()
            assert np.array_equal(cg, cr), "cells differ at generation %d" % g
            assert np.array_equal(ag, ar), "alive set differs at generation %d" % g
    st = gpu.heap.stats()
    assert st["error_flags"] == 0
    check_invariants(gpu.heap, [W * H, ref.alive_count()])
    return gpu, ref


def test_life_64x64_100_generations_bit_exact():
    # the 64x64, density 0.25, 100-generation workload
    _run_pair(64, 64, WL.gol_initial(64, 64, 1), 100)


@pytest.mark.parametrize("W,H,seed,gens", [(3, 3, 2, 12), (37, 5, 3, 60), (200, 130, 4, 40)])
def test_life_ragged_grids(W, H, seed, gens):
    _run_pair(W, H, WL.gol_initial(W, H, seed), gens, full_every=5)


def test_empty_and_full_grids():
    _run_pair(16, 16, np.zeros((16, 16), np.uint8), 3)
    _run_pair(16, 16, np.ones((16, 16), np.uint8), 3)


def test_glider_wraps_torus():
    g = np.zeros((64, 64), np.uint8)
    for x, y in [(1, 0), (2, 1), (0, 2), (1, 2), (2, 2)]:
        g[y, x] = 1
    gpu, _ = _run_pair(64, 64, g, 256, full_every=64)
    _, alive = gpu.dump()
    assert sorted(map(tuple, alive)) == sorted([(1, 0), (2, 1), (0, 2), (1, 2), (2, 2)])


def test_life_large_grid_hash_parity():
    # 1024 x 1024: every generation's state hash matches; blocks churn heavily
    _run_pair(1024, 1024, WL.gol_initial(1024, 1024, 5), 30, full_every=15)
