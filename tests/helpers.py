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


def expected_stats(snap):
    """Block and object counts of a quiescent heap snapshot from the block
    states of Fig. 2: a block is free iff its bit in the free bitmap is set
    (a free block and a full one both have no free slot in their object
    bitmap); a non-free block of type T is allocated[T], and active[T] if it
    has a free slot. Live objects are the occupied slots of the allocated
    blocks. The oracle's checker first confirms the snapshot's bitmaps agree
    with the object bitmaps (I1-I5); its live counts must equal these."""
    bad, live = O.check_heap(**snap)
    assert bad == 0, "heap invariants violated: bits %d" % bad
    M = int(snap["M"])
    width = int(snap["width"])
    cap = snap["capacity"].astype(np.int64)
    obj = snap["obj_free"]
    bt = snap["block_type"].astype(np.int64)
    b = np.arange(M)
    leaf = snap["free_bm"][: int(snap["words_per_level"][0])]
    free = ((leaf[b // width] >> (b % width).astype(np.uint64)) & np.uint64(1)).astype(bool)
    free_slots = np.array([bin(int(w)).count("1") for w in obj], dtype=np.int64)
    n_types = len(cap)
    out = {"free_blocks": int(free.sum()), "allocated_blocks": [0] * n_types, "active_blocks": [0] * n_types,
           "live_objects": [0] * n_types}
    for t in range(n_types):
        mine = (bt == t) & ~free
        out["live_objects"][t] = int((cap[t] - free_slots[mine]).sum())
        out["allocated_blocks"][t] = int(mine.sum())
        out["active_blocks"][t] = int((mine & (free_slots > 0)).sum())
    assert out["live_objects"] == [int(x) for x in live]
    return out


def check_stats(heap):
    """dsr_heap_stats of a quiescent heap equals expected_stats of its snapshot; returns the stats."""
    exp = expected_stats(heap.snapshot())
    st = heap.stats()
    for k in ("free_blocks", "allocated_blocks", "active_blocks", "live_objects"):
        assert st[k] == exp[k], (k, st[k], exp[k])
    return st
