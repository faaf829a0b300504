"""Do-alls over a type with subtypes (Section 1: class inheritance without
wasted memory; Section 2.3 do-all): a do-all over a base type visits the
live objects of the base and of every subtype, each method call sees the
object's concrete type, and objects keep their own type's block layout.

The expected results are the built-in methods' definitions applied to the
dumps of each concrete type; the block-state invariants are checked with the
oracle's checker."""
import numpy as np
import pytest
import torch

from paper_1809_07444_gb300 import _lib as L
from paper_1809_07444_gb300.heap import Heap, heap_bytes_for_blocks

from helpers import check_invariants

pytestmark = pytest.mark.gpu

# Base {a}; D1 : Base {a, b}; D2 : Base {a, c (8 bytes)}; D3 : D1 {a, b, d}
TYPES = [[4], [4, 4], [4, 8], [4, 4, 4]]
BASES = [-1, 0, 0, 1]
SUB = [[0, 1, 2, 3], [1, 3], [2], [3]]


def _heap(n_objects=60_000, seed=7):
    h = Heap(TYPES, heap_bytes_for_blocks(TYPES, 8000), bases=BASES)
    refs = torch.empty(n_objects, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 4, seed)  # type drawn per object, field 0 = object index
    return h


def _by_handle(h, t):
    f, hd = h.dump(t)
    o = np.argsort(hd)
    return f[o].view(np.int32), hd[o]


def test_do_all_over_a_type_visits_its_subtree():
    h = _heap()
    live = check_invariants(h)
    assert min(live) > 1000  # every type has objects
    for t in range(4):
        assert h.count(t) == sum(live[u] for u in SUB[t])
    # dumps stay per concrete type
    for t in range(4):
        assert len(h.dump(t)[0]) == live[t]
    assert h.stats()["error_flags"] == 0


def test_stream_add_over_a_mid_level_type_uses_each_concrete_layout():
    # D1 (2 fields, 32 slots a block) and D3 (3 fields, 20 slots a block)
    # share one do-all of 32 threads per listed block
    h = _heap(seed=9)
    before = {t: _by_handle(h, t) for t in range(4)}
    h.parallel_do(1, L.METHOD_STREAM_ADD, None)
    for t in range(4):
        f1, hd1 = _by_handle(h, t)
        f0, hd0 = before[t]
        assert np.array_equal(hd0, hd1)
        if t in SUB[1]:
            k = f0.shape[1]
            want = f0.copy()
            for f in range(k - 1):
                want[:, f] = f0[:, f] + f0[:, f + 1]
            want[:, k - 1] = f0[:, k - 1] + 1
            assert np.array_equal(f1, want), t
        else:
            assert np.array_equal(f1, f0), t  # outside the subtree: untouched
    assert h.stats()["error_flags"] == 0


def test_method_that_needs_4_byte_fields_is_refused_over_a_subtree_with_wider_fields():
    h = _heap()
    with pytest.raises(L.DsrError):
        h.parallel_do(0, L.METHOD_STREAM_ADD, None)  # D2 has an 8-byte field
    h.parallel_do(3, L.METHOD_STREAM_ADD, None)  # a leaf type alone is fine
    assert h.stats()["error_flags"] == 0


def test_delete_inside_a_do_all_over_the_base():
    h = _heap(seed=11)
    live = check_invariants(h)
    a0 = {t: _by_handle(h, t)[0][:, 0] for t in range(4)}
    h.parallel_do(0, L.METHOD_DELETE_IF, L.DeleteIfArgs(3, 1))
    want = [int((a0[t] % 3 != 1).sum()) for t in range(4)]
    live2 = check_invariants(h, want)
    for t in range(4):
        a = _by_handle(h, t)[0][:, 0]
        assert (a % 3 != 1).all()
        assert np.array_equal(np.sort(a), np.sort(a0[t][a0[t] % 3 != 1]))
    assert h.count(0) == sum(live2) and list(live2) != list(live)
    assert h.stats()["error_flags"] == 0


def test_clone_out_of_a_subtree_visits_only_the_objects_live_at_the_start():
    h = _heap(seed=13)
    live = check_invariants(h)
    with pytest.raises(L.DsrError):
        h.parallel_do(1, L.METHOD_CLONE, L.CloneArgs(3, 0))  # D3 lies inside D1's subtree
    a1 = np.concatenate([_by_handle(h, t)[0][:, 0] for t in SUB[1]])
    base_before = _by_handle(h, 0)[0][:, 0]
    h.parallel_do(1, L.METHOD_CLONE, L.CloneArgs(0, 5_000_000))  # copies of D1 and D3 objects as Base
    base_after = _by_handle(h, 0)[0][:, 0]
    want = np.sort(np.concatenate([base_before, a1 + 5_000_000]))
    assert np.array_equal(np.sort(base_after), want)
    check_invariants(h, [live[0] + live[1] + live[3], live[1], live[2], live[3]])
    assert h.stats()["error_flags"] == 0


def test_without_bases_a_do_all_visits_one_type():
    h = Heap(TYPES, heap_bytes_for_blocks(TYPES, 8000))
    refs = torch.empty(20_000, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 4, 3)
    live = check_invariants(h)
    assert [h.count(t) for t in range(4)] == list(live)
    h.set_bases(BASES)
    assert h.count(0) == sum(live)
