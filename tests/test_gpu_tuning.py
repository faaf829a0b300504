"""Tuning knobs change speed, never results: game of life, wa-tor (plain and
batched) and the allocator under every value of threads, cap_min and bitmap
fan-out match the oracle bit for bit, with consistent heaps."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1809_07444_gb300 import autotune as AT
from paper_1809_07444_gb300 import workloads as WL
from paper_1809_07444_gb300.apps import Gol, Wator, WatorBatch
from paper_1809_07444_gb300.heap import Heap, heap_bytes_for_blocks

from helpers import check_invariants, check_stats

pytestmark = pytest.mark.gpu

TUNINGS = [
    {"threads": 128, "cap_min": 32, "fanout": 16},
    {"threads": 512, "cap_min": 64, "fanout": 32},
    {"threads": 64, "cap_min": 32, "fanout": 64},
    {"threads": 1024, "cap_min": 64, "fanout": 16},
]


@pytest.mark.parametrize("tun", TUNINGS)
def test_life_under_tuning(tun):
    start = WL.gol_initial(64, 64, 1)
    gpu, ref = Gol(64, 64, start, tuning=tun), O.Gol(64, 64, start)
    assert gpu.heap.layout().fanout == tun["fanout"]
    for g in range(1, 41):
        gpu.step(1)
        ref.step(1)
        assert gpu.hash() == ref.hash(), "generation %d" % g
    cg, ag = gpu.dump()
    cr, ar = ref.dump()
    assert np.array_equal(cg, cr) and np.array_equal(ag, ar)
    assert gpu.heap.stats()["error_flags"] == 0
    check_invariants(gpu.heap, [64 * 64, ref.alive_count()])


@pytest.mark.parametrize("tun", TUNINGS)
def test_wator_under_tuning(tun):
    W, H = 96, 80
    k0 = WL.wator_initial(W, H, 6)
    gpu, ref = Wator(W, H, k0, 6, tuning=tun), O.Wator(W, H, k0, seed=6)
    for t in range(1, 61):
        gpu.step(1)
        ref.step(1)
        assert gpu.hash() == ref.hash(), "step %d" % t
    fg, sg = gpu.dump()
    fr, sr = ref.dump()
    assert np.array_equal(fg, fr) and np.array_equal(sg, sr)
    assert gpu.heap.stats()["error_flags"] == 0
    check_invariants(gpu.heap, list(ref.counts()))
    # dsr_heap_stats at this fan-out: its live counts are the oracle's
    assert tuple(gpu.counts()) == tuple(ref.counts())
    check_stats(gpu.heap)


@pytest.mark.parametrize("tun", TUNINGS[:2])
def test_batched_wator_under_tuning(tun):
    sides = [17, 40, 64, 5, 90]
    b = WatorBatch(192 << 20, max_instances=8, tuning=tun)
    refs, slots = [], []
    for i, s in enumerate(sides):
        k0 = WL.wator_initial(s, s, 300 + i)
        slots.append(b.add(s, s, k0, 300 + i))
        refs.append(O.Wator(s, s, k0, seed=300 + i))
    for t in range(1, 31):
        b.step(1)
        for slot, ref in zip(slots, refs):
            ref.step(1)
            assert b.hash(slot) == ref.hash(), "instance %d, step %d" % (slot, t)
    for slot, ref in zip(slots, refs):
        hp = b.heap(slot)
        assert hp.layout().fanout == tun["fanout"]
        assert hp.stats()["error_flags"] == 0
        check_invariants(hp, list(ref.counts()))
        assert tuple(b.counts(slot)) == tuple(ref.counts())
        check_stats(hp)


@pytest.mark.parametrize("fanout", [32, 16])
def test_allocator_many_levels_narrow_fanout(fanout):
    # 70,000 blocks: 4 levels at fan-out 32, 5 at 16
    types = [[4, 4], [4, 4, 4, 4]]
    tun = {"fanout": fanout}
    h = Heap(types, heap_bytes_for_blocks(types, 70_000, tun), tuning=tun)
    assert h.layout().n_levels == (4 if fanout == 32 else 5)
    n = 1_000_000
    refs = torch.empty(n, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 2, 3)
    live = check_invariants(h)
    assert live.sum() == n
    assert sum(check_stats(h)["live_objects"]) == n
    r = refs.cpu().numpy().view(np.uint64)
    assert len(np.unique(r)) == n
    from paper_1809_07444_gb300 import _lib as L
    h.parallel_do(0, L.METHOD_DELETE_IF, L.DeleteIfArgs(3, 1))
    check_invariants(h)
    check_stats(h)
    for t in range(2):
        h.parallel_do(t, L.METHOD_DELETE_IF, L.DeleteIfArgs(1, 0))  # everything left
    st = h.stats()
    assert st["error_flags"] == 0 and st["free_blocks"] == st["n_blocks"]
    check_invariants(h, [0, 0])


def test_autotuner_picks_a_runnable_setting_on_a_small_batch():
    sides, seeds = [32, 48, 64, 20], [1, 2, 3, 4]
    space = {"threads": [128, 256], "cap_min": [64, 32], "fanout": [64, 16]}
    best, v, table = AT.search(AT.wator_batch_measure(sides, seeds, steps=3, warmup=1), space)
    assert v > 0 and all(best[k] in space[k] for k in space)
    assert all(x is not None and x > 0 for x in table.values())


@pytest.mark.parametrize("fanout", [64, 32, 16])
def test_heap_stats_match_block_states_at_every_fanout(fanout):
    # dsr_heap_stats against the counts the block states of Fig. 2 give for
    # the same snapshot, on a block count that is not a multiple of
    # 64 * fanout (a ragged last leaf word), after allocation, churn and
    # partial and complete deletion
    import ctypes as C

    from paper_1809_07444_gb300 import _lib as L

    types = [[4, 4], [4, 4, 4, 4], [4]]
    tun = {"fanout": fanout}
    h = Heap(types, heap_bytes_for_blocks(types, 8192 + 777, tun), tuning=tun)
    M = h.layout().n_blocks
    assert M >= 8192 + 777 and M % (64 * fanout) != 0
    n = 90_000
    refs = torch.empty(n, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 3, 11)
    st = check_stats(h)
    assert sum(st["live_objects"]) == n and st["error_flags"] == 0
    replaced = torch.zeros(1, dtype=torch.int64, device="cuda")
    L.check(h.lib.dsr_bench_churn(h.handle, n, 3, 12, C.c_void_p(refs.data_ptr()), C.c_void_p(replaced.data_ptr()),
                                  None), "dsr_bench_churn")
    st = check_stats(h)
    assert sum(st["live_objects"]) == n and int(replaced.item()) > 0
    h.parallel_do(1, L.METHOD_DELETE_IF, L.DeleteIfArgs(3, 1))
    check_stats(h)
    for t in range(3):
        h.parallel_do(t, L.METHOD_DELETE_IF, L.DeleteIfArgs(1, 0))
    st = check_stats(h)
    assert st["free_blocks"] == M and st["live_objects"] == [0, 0, 0] and st["error_flags"] == 0
