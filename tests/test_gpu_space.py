"""Space-efficiency search (Section 4, Fig. 8): the largest wa-tor side that a
fixed heap runs without running out of memory."""
import pytest

import oracle as O
from paper_1809_07444_gb300 import space
from paper_1809_07444_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def test_max_side_fits_and_the_next_sizes_do_not():
    heap, steps = 2 << 20, 30
    side, peak = space.max_wator_side(heap, steps)
    assert side > 16
    assert 0 < peak <= heap
    # The live objects of a run are the simulation's, but where concurrent
    # allocations put them (how full each block ends up) depends on
    # scheduling, so at the largest side a second run may or may not fit.
    # A few percent below it every run fits, with the same peak live bytes.
    below = int(side * 0.97)
    ok, peak1 = space.wator_fits(below, heap, steps)
    ok2, peak2 = space.wator_fits(below, heap, steps)
    assert ok and ok2 and peak1 == peak2 and 0 < peak1 < peak
    for tun in ({"fanout": 16}, {"fanout": 32, "cap_min": 32}):
        ok3, peak3 = space.wator_fits(below, heap * 2, steps, tuning=tun)
        assert ok3 and peak3 == peak1  # live counts do not depend on the fan-out
    # a clearly larger torus does not fit the same heap
    assert not space.wator_fits(int(side * 1.25) + 2, heap, steps)[0]


def test_smaller_blocks_hold_at_least_as_large_a_problem():
    heap, steps = 2 << 20, 30
    s64, _ = space.max_wator_side(heap, steps)
    s32, _ = space.max_wator_side(heap, steps, tuning={"cap_min": 32})
    assert s32 >= s64 * 0.95  # 32-slot blocks waste no more space at the ends of runs


def test_experiment_reports_every_setting():
    out = space.experiment(heap_bytes=1 << 20, steps=10)
    rows = out["rows"]
    assert [r["tuning"] for r in rows[:3]] == ["default", {"cap_min": 32}, {"fanout": 16}]
    assert [r["allocator"] for r in rows] == ["dsr"] * 3 + ["BitmapAlloc"] * 2
    assert all(r["max_side"] > 0 and 0 < r["efficiency"] <= 1 for r in rows)
    # every row's peak live bytes is the oracle's peak over the same run
    # (the live counts come from dsr_heap_stats, at fan-out 64 and 16)
    for r in rows:
        side = r["max_side"]
        ref = O.Wator(side, side, WL.wator_initial(side, side, 1), seed=1)
        peak = 0
        for _ in range(out["steps"]):
            ref.step(1)
            f, sh = ref.counts()
            peak = max(peak, f * space.OBJECT_BYTES[0] + sh * space.OBJECT_BYTES[1])
        assert r["peak_live_bytes"] == peak, (r, peak)
        assert r["efficiency"] == peak / out["heap_bytes"]


def test_bitmap_capacities_fill_the_heap():
    heap = 8 << 20
    cf, cs = space.bitmap_capacities(heap, 0.8)
    assert cf % 64 == 0 and cs % 64 == 0
    used = cf * 12 + cs * 16
    assert 0.97 * heap < used <= heap
