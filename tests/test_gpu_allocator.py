"""GPU tests of the device allocator and the do-all (Alg. 1, Alg. 2, Section 2.3).

Every test checks the block-state invariants with the oracle's checker at
quiescent points, and compares live-object sets with what the operations
imply (the allocator's placement is free; only the set of objects is fixed).
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1809_07444_gb300 import _lib as L
from paper_1809_07444_gb300.heap import Heap, heap_bytes_for_blocks

from helpers import check_invariants

pytestmark = pytest.mark.gpu

TYPES3 = [[4, 4], [4, 4, 4], [4, 4, 4, 4, 4, 4, 4, 4]]  # capacities 64, 42, 16


def _heap(n_blocks, types=TYPES3, **kw):
    return Heap(types, heap_bytes_for_blocks(types, n_blocks, kw.get("tuning")), **kw)


def _expected_types(n, n_types, seed):
    # type draw of the allocation kernel: mix64(seed ^ (i * GAMMA)) mod n_types
    import oracle as O
    G = 0x9E3779B97F4A7C15
    return np.array([O.mix64(seed ^ ((i * G) & 0xFFFFFFFFFFFFFFFF)) % n_types for i in range(n)])


def test_fresh_heap_is_all_free():
    h = _heap(5000)
    st = h.stats()
    assert st["free_blocks"] == st["n_blocks"] >= 5000
    assert st["error_flags"] == 0
    check_invariants(h, [0, 0, 0])


@pytest.mark.parametrize("n,n_types", [(1, 1), (31, 1), (1000, 3), (200_003, 3)])
def test_alloc_then_free_everything(n, n_types):
    h = _heap(20000)
    refs = torch.empty(n, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, n_types, 12345)
    torch.cuda.synchronize()
    r = refs.cpu().numpy().view(np.uint64)
    assert (r != np.uint64(L.NULL_REF)).all()
    assert len(np.unique(r)) == n  # I6: no slot handed out twice
    want_t = _expected_types(n, n_types, 12345) if n <= 1000 else None
    live = check_invariants(h)
    assert live.sum() == n
    st = h.stats()
    assert st["error_flags"] == 0
    # each object holds its thread index in field 0
    tid = []
    for t in range(n_types):
        f, hd = h.dump(t)
        tid.append(f[:, 0].astype(np.int64))
        assert len(f) == live[t]
        if want_t is not None:
            assert np.array_equal(np.sort(f[:, 0]), np.nonzero(want_t == t)[0])
    assert np.array_equal(np.sort(np.concatenate(tid)), np.arange(n))
    # dense placement: allocation-only, so blocks are nearly full; the slack
    # comes from concurrent leaders (at most one slow path per SM per type
    # at a time)
    for t in range(n_types):
        need = -(-live[t] // st["capacity"][t])
        assert st["allocated_blocks"][t] <= 2 * need + 4 * 152
        if live[t] >= 50_000:
            fill = live[t] / (st["allocated_blocks"][t] * st["capacity"][t])
            assert fill >= 0.5, fill
    h.bench_free(refs)
    st = h.stats()
    assert st["error_flags"] == 0
    assert st["free_blocks"] == st["n_blocks"]
    check_invariants(h, [0] * 3)


def test_repeated_alloc_free_cycles_reuse_blocks():
    h = _heap(8000)
    refs = torch.empty(100_000, dtype=torch.int64, device="cuda")
    for cyc in range(5):
        h.bench_alloc(refs, 3, cyc)
        h.bench_free(refs)
    st = h.stats()
    assert st["error_flags"] == 0 and st["free_blocks"] == st["n_blocks"]
    check_invariants(h, [0, 0, 0])


def test_out_of_memory_is_reported_not_hung():
    h = _heap(100, types=[[4, 4]])
    st0 = h.stats()
    cap = st0["n_blocks"] * 64
    refs = torch.empty(cap + 5000, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 1, 7)
    torch.cuda.synchronize()
    r = refs.cpu().numpy().view(np.uint64)
    ok = (r != np.uint64(L.NULL_REF)).sum()
    assert ok == cap
    st = h.stats()
    assert st["error_flags"] & L.ERR_OOM
    assert st["free_blocks"] == 0
    check_invariants(h, [cap])


def test_injected_slow_path_failures():
    h = _heap(1000, types=[[4, 4]])
    h.inject_oom(3)
    refs = torch.empty(64 * 10, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 1, 9)
    torch.cuda.synchronize()
    r = refs.cpu().numpy().view(np.uint64)
    st = h.stats()
    assert st["error_flags"] & L.ERR_OOM
    n_ok = int((r != np.uint64(L.NULL_REF)).sum())
    assert 0 < n_ok < len(r)
    check_invariants(h, [n_ok])


def test_doall_visits_live_set_snapshot():
    h = _heap(4000)
    refs = torch.empty(50_000, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 2, 3)
    live = check_invariants(h)
    assert h.count(0) == live[0] and h.count(1) == live[1]
    # delete the objects of type 0 whose field0 is even, inside a do-all
    h.parallel_do(0, L.METHOD_DELETE_IF, L.DeleteIfArgs(2, 0))
    f0, _ = h.dump(0)
    assert (f0[:, 0] % 2 == 1).all()
    live2 = check_invariants(h)
    assert live2[0] == len(f0) and live2[1] == live[1]
    # a do-all over type 1 that creates type-2 copies: the copies exist, the
    # do-all saw only the type-1 objects that were live when it started
    h.parallel_do(1, L.METHOD_CLONE, L.CloneArgs(2, 1000000))
    f1, _ = h.dump(1)
    f2, _ = h.dump(2)
    assert len(f2) == len(f1)
    assert np.array_equal(np.sort(f2[:, 0].astype(np.int64)), np.sort(f1[:, 0].astype(np.int64)) + 1000000)
    assert h.stats()["error_flags"] == 0
    check_invariants(h, [live2[0], live[1], len(f1)])


def test_clone_into_same_type_family_is_not_revisited():
    # objects created by a do-all over type 0 into type 1, then a do-all over 1
    # into 0: each round visits exactly the objects live at its start
    h = _heap(3000, types=[[4, 4], [4, 4]])
    refs = torch.empty(10_000, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 1, 5)
    n0 = 10_000
    h.parallel_do(0, L.METHOD_CLONE, L.CloneArgs(1, 0))
    assert h.count(1) == n0
    h.parallel_do(1, L.METHOD_CLONE, L.CloneArgs(0, 0))
    assert h.count(0) == 2 * n0
    check_invariants(h, [2 * n0, n0])


def test_churn_mixed_delete_and_new_in_one_kernel():
    # a do-all deletes half of type A while another do-all's new objects
    # reuse the freed slots; repeated, the heap stays consistent and dense
    h = _heap(6000, types=[[4, 4], [4, 4, 4]])
    refs = torch.empty(150_000, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 2, 11)
    for rnd in range(6):
        h.parallel_do(0, L.METHOD_DELETE_IF, L.DeleteIfArgs(3, rnd % 3))
        h.parallel_do(1, L.METHOD_CLONE, L.CloneArgs(0, rnd + 1))
        h.parallel_do(1, L.METHOD_DELETE_IF, L.DeleteIfArgs(4, rnd % 4))
        live = check_invariants(h)
        assert h.count(0) == live[0] and h.count(1) == live[1]
    assert h.stats()["error_flags"] == 0


@pytest.mark.parametrize("types,t,holes", [
    ([[4, 4, 4, 4]], 0, False),          # 128-bit vector path, full quads
    ([[4, 4, 4, 4]], 0, True),           # vector path, partly live quads
    ([[4], [4] * 8], 1, True),           # vector path, 8 fields, capacity 8
    ([[4, 4], [4, 4, 4]], 1, True),      # capacity 42: scalar path
    ([[4, 4]], 0, True),                 # 2 fields
])
def test_stream_add_method_updates_every_field(types, t, holes):
    h = _heap(6000, types=types)
    refs = torch.empty(40_000, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, len(types), 2)
    if holes:
        h.parallel_do(t, L.METHOD_DELETE_IF, L.DeleteIfArgs(3, 1))
    _check_stream_add(h, t)


def _check_stream_add(h, t):
    f_before, hd = h.dump(t)
    order = np.argsort(hd)
    f_before = f_before[order].view(np.int32)
    h.parallel_do(t, L.METHOD_STREAM_ADD, None)
    f_after, hd2 = h.dump(t)
    f_after = f_after[np.argsort(hd2)].view(np.int32)
    assert np.array_equal(np.sort(hd), np.sort(hd2))  # same objects, nothing moved
    k = f_before.shape[1]
    want = f_before.copy()  # int32 arithmetic wraps like the kernel's
    for f in range(k - 1):
        want[:, f] = f_before[:, f] + f_before[:, f + 1]
    want[:, k - 1] = f_before[:, k - 1] + 1
    assert np.array_equal(f_after, want)
    assert h.stats()["error_flags"] == 0


def test_three_level_bitmaps_stay_consistent():
    # M > 64^2 blocks: three bitmap levels; allocate enough to touch many
    # containers, free a scattered subset, then everything
    h = _heap(70_000, types=[[4, 4]])
    assert h.layout().n_levels == 3
    n = 64 * 30_000
    refs = torch.empty(n, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 1, 1)
    check_invariants(h, [n])
    h.parallel_do(0, L.METHOD_DELETE_IF, L.DeleteIfArgs(7, 3))
    check_invariants(h, [n - len(range(3, n, 7))])
    h.parallel_do(0, L.METHOD_DELETE_IF, L.DeleteIfArgs(1, 0))
    st = h.stats()
    assert st["free_blocks"] == st["n_blocks"] and st["error_flags"] == 0
    check_invariants(h, [0])


def test_churn_kernel_replaces_half_and_keeps_the_heap_consistent():
    # deletes and creates interleaved in one kernel: the live set is the
    # thread indices again (replacements hold the same index)
    h = _heap(20000)
    n = 200_000
    refs = torch.empty(n, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 3, 21)
    nrep = torch.zeros(1, dtype=torch.int64, device="cuda")
    L.check(h.lib.dsr_bench_churn(h.handle, n, 3, 99, C.c_void_p(refs.data_ptr()), C.c_void_p(nrep.data_ptr()),
                                  None), "dsr_bench_churn")
    torch.cuda.synchronize()
    import oracle as O
    G = 0x9E3779B97F4A7C15
    want = sum(O.mix64(99 ^ ((i * G) & 0xFFFFFFFFFFFFFFFF)) & 1 for i in range(n))
    assert int(nrep.item()) == want
    r = refs.cpu().numpy().view(np.uint64)
    assert (r != np.uint64(L.NULL_REF)).all() and len(np.unique(r)) == n
    live = check_invariants(h)
    assert live.sum() == n
    ids = np.concatenate([h.dump(t)[0][:, 0].astype(np.int64) for t in range(3)])
    assert np.array_equal(np.sort(ids), np.arange(n))
    h.bench_free(refs)
    st = h.stats()
    assert st["error_flags"] == 0 and st["free_blocks"] == st["n_blocks"]


def test_fma_probe_runs():
    out = torch.empty(4 * 256, dtype=torch.float32, device="cuda")
    L.check(L.load().dsr_bench_fma(C.c_void_p(out.data_ptr()), 4, 1000, None), "dsr_bench_fma")
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()


def test_atomic_probe_leaves_each_word_as_its_last_atomic_set_it():
    words = torch.zeros(1000, dtype=torch.int64, device="cuda")
    lib = L.load()
    L.check(lib.dsr_bench_atomics(C.c_void_p(words.data_ptr()), 1000, 5, 0, None), "dsr_bench_atomics")
    torch.cuda.synchronize()
    # 5 atomics: or, and, or, and, or -> each thread's own bit set
    want = np.array([1 << (i % 64) for i in range(1000)], dtype=np.uint64)
    assert np.array_equal(words.cpu().numpy().view(np.uint64), want)
    L.check(lib.dsr_bench_atomics(C.c_void_p(words.data_ptr()), 1000, 8, 1, None), "dsr_bench_atomics")
    torch.cuda.synchronize()


def test_delete_of_a_slot_beyond_capacity_is_rejected():
    # type 1 has capacity 42: a handle with slot 50 is not a slot of it
    h = _heap(100, types=[[4, 4], [4, 4, 4]])
    refs = torch.empty(64, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 2, 1)
    assert h.stats()["capacity"][1] == 42
    f1, hd1 = h.dump(1)
    bid = int(hd1[0]) >> 6
    bad = torch.tensor([np.int64((bid << 6) | 50), np.int64(-1)], dtype=torch.int64, device="cuda")
    h.bench_free(bad)
    st = h.stats()
    assert st["error_flags"] & L.ERR_BAD_HANDLE
    check_invariants(h)  # nothing else changed
    assert h.count(1) == len(f1)
