"""Subtype declarations (Section 1: class inheritance without wasted memory),
host side: the hierarchy checks of dsr_type_tree and the per-type block
geometry of a hierarchy (no CUDA call)."""
import ctypes as C

import pytest

from paper_1809_07444_gb300 import _lib as L
from paper_1809_07444_gb300.heap import _descs, type_tree

# Base {a}; D1 : Base {a, b}; D2 : Base {a, c (8 bytes)}; D3 : D1 {a, b, d}
TYPES = [[4], [4, 4], [4, 8], [4, 4, 4]]
BASES = [-1, 0, 0, 1]


def test_subtree_masks():
    assert type_tree(TYPES, BASES) == [0b1111, 0b1010, 0b0100, 0b1000]
    assert type_tree(TYPES, [-1] * 4) == [1, 2, 4, 8]


def test_chain_masks_are_transitive():
    types = [[4], [4, 4], [4, 4, 4], [4, 4, 4, 4]]
    assert type_tree(types, [-1, 0, 1, 2]) == [0b1111, 0b1110, 0b1100, 0b1000]


@pytest.mark.parametrize("types,bases", [
    (TYPES, [-1, 0, 0, 3]),            # a base declared after its subtype
    (TYPES, [-1, 0, 0, 7]),            # base index out of range
    (TYPES, [-2, 0, 0, 1]),            # below -1
    ([[4], [8, 4]], [-1, 0]),          # leading field size differs from the base's
    ([[4, 4], [4]], [-1, 0]),          # subtype with fewer fields than its base
    ([[4, 8], [4, 4, 8]], [-1, 0]),    # second inherited field differs
])
def test_invalid_hierarchies_are_rejected(types, bases):
    with pytest.raises(L.DsrError):
        type_tree(types, bases)


def test_each_subtype_gets_blocks_sized_for_itself():
    # "without wasted memory": a block of type T holds floor(64 * s_min / s_T)
    # objects of T's own size (Section 2, block capacities), so base objects
    # are not padded to the largest subtype and subtypes carry only their
    # own fields
    lib = L.load()
    descs, _keep = _descs(TYPES)
    lay = L.Layout()
    L.check(lib.dsr_heap_plan(descs, len(TYPES), 1000, None, C.byref(lay)), "dsr_heap_plan")
    def soa_bytes(t, c):  # each field's SOA array starts on an 8-byte boundary
        return sum((c * b + 7) // 8 * 8 for b in TYPES[t])

    assert lay.block_bytes == 256  # 64 slots of the 4-byte base type
    for t, fields in enumerate(TYPES):
        c = lay.capacity[t]
        limit = min(64, 64 * 4 // sum(fields))
        assert c <= limit and soa_bytes(t, c) <= lay.block_bytes
        assert c == limit or soa_bytes(t, c + 1) > lay.block_bytes  # as many as fit
    assert [lay.capacity[t] for t in range(4)] == [64, 32, 21, 20]
