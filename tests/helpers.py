"""Shared test helpers: heap invariants via the oracle's checker."""
import numpy as np

import oracle as O


def check_invariants(heap, expect_live=None):
    """Assert I1-I5 (and I7 if expect_live is given) on a quiescent GPU heap; returns live counts."""
    snap = heap.snapshot()
    bad, live = O.check_heap(**snap)
    assert bad == 0, "heap invariants violated: bits %d" % bad
    if expect_live is not None:
        assert list(live) == list(expect_live), (list(live), list(expect_live))
    return live


def rows_equal(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return a.shape == b.shape and np.array_equal(a, b)
