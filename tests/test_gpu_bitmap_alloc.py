"""The BitmapAlloc comparator (flat per-type bitmap, AOS objects) runs the
same wa-tor rules and matches the oracle step by step."""
import pytest

import oracle as O
from paper_1809_07444_gb300 import _lib as L
from paper_1809_07444_gb300 import workloads as WL
from paper_1809_07444_gb300.apps import Wator, WatorBitmap

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W,H,seed,steps", [(64, 64, 1, 120), (17, 9, 3, 80), (257, 129, 4, 40)])
def test_bitmap_alloc_wator_matches_oracle(W, H, seed, steps):
    k0 = WL.wator_initial(W, H, seed)
    bm, ref, dyn = WatorBitmap(W, H, k0, seed), O.Wator(W, H, k0, seed=seed), Wator(W, H, k0, seed)
    assert bm.hash() == ref.hash()
    for t in range(1, steps + 1):
        bm.step(1)
        ref.step(1)
        dyn.step(1)
        assert bm.hash() == ref.hash(), "step %d" % t
        assert bm.counts() == ref.counts()
    st = bm.heap.stats()
    assert st["error_flags"] == 0
    # the same allocations, frees and moves as the dsr heap (visits differ
    # here by the hash do-alls run on the comparator only)
    cb, cd = bm.heap.counters(), dyn.heap.counters()
    assert (cb["allocs"], cb["frees"], cb["app0"]) == (cd["allocs"], cd["frees"], cd["app0"])


def test_bitmap_alloc_visits_equal_the_dsr_form():
    k0 = WL.wator_initial(96, 96, 5)
    bm, dyn = WatorBitmap(96, 96, k0, 5), Wator(96, 96, k0, 5)
    bm.step(30)
    dyn.step(30)
    assert bm.heap.counters()["visits"] == dyn.heap.counters()["visits"] > 0


def test_bitmap_alloc_full_size():
    W = H = 2048
    k0 = WL.wator_initial(W, H, 1)
    bm, ref = WatorBitmap(W, H, k0, 1), O.Wator(W, H, k0, seed=1)
    for t in range(1, 21):
        bm.step(1)
        ref.step(1)
        assert bm.hash() == ref.hash(), "step %d" % t


def test_bitmap_alloc_out_of_memory_is_reported():
    # room for the initial fish only: births fail and raise DSR_ERR_OOM
    W = H = 64
    k0 = WL.wator_initial(W, H, 2)
    n_fish = int((k0 == 1).sum())
    bm = WatorBitmap(W, H, k0, 2, capacity=[-(-n_fish // 64) * 64, 4096])
    bm.step(10)
    assert bm.heap.stats()["error_flags"] & L.ERR_OOM
