"""Oracle pins: counter generator, object hash, hierarchical bitmap (Section 3, Alg. 2, Fig. 5)."""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_splitmix64_published_outputs():
    for seed, idx, val in _rows("splitmix64.txt"):
        assert O.splitmix_at(int(seed), int(idx)) == int(val)


def test_rand_composes_streams_steps_cells():
    # Every coordinate of the counter changes the output, and draws are
    # close to uniform over 4 choices (chi-square, 3 dof, p ~ 1e-6 bound).
    base = O.rand(7, 0, 3, 100)
    assert base != O.rand(8, 0, 3, 100)
    assert base != O.rand(7, 1, 3, 100)
    assert base != O.rand(7, 0, 4, 100)
    assert base != O.rand(7, 0, 3, 101)
    n = 40000
    counts = np.bincount([O.rand(1, 0, 0, c) % 4 for c in range(n)], minlength=4)
    chi2 = ((counts - n / 4) ** 2 / (n / 4)).sum()
    assert chi2 < 30.0


def test_obj_hash_sensitive_to_type_order_and_value():
    h = O.obj_hash(0, [1, 2, 3])
    assert h != O.obj_hash(1, [1, 2, 3])
    assert h != O.obj_hash(0, [2, 1, 3])
    assert h != O.obj_hash(0, [1, 2, 4])
    assert h != O.obj_hash(0, [1, 2])
    # negative values hash by their 32-bit pattern
    assert O.obj_hash(0, [-1]) == O.obj_hash(0, [0xFFFFFFFF])


def test_fig5_worked_example():
    g = {r[0]: r[1:] for r in _rows("fig5_hier_bitmap.txt")}
    hb = O.HierBitmap(int(g["N"][0]), width=int(g["width"][0]))
    assert hb.levels == int(g["levels"][0])
    for b in g["set"]:
        ok, _ = hb.try_set(int(b))
        assert ok
    assert hb.consistent()
    ok, trace = hb.try_clear(int(g["clear"][0]))
    assert ok
    want = [tuple(int(v) for v in t.split(":")) for t in g["trace"]]
    assert trace == want
    assert hb.consistent()
    # clearing the same bit again fails and changes nothing
    ok, trace = hb.try_clear(int(g["clear"][0]))
    assert not ok and trace == []


def _nested_from_flat(flat, width, level):
    """Bit i of `level` is set iff a flat bit lies in [i*width^level, (i+1)*width^level)."""
    span = width ** level
    n = -(-len(flat) // span)
    return np.array([flat[i * span:(i + 1) * span].any() for i in range(n)], dtype=np.uint8)


@pytest.mark.parametrize("width,n_bits", [(4, 32), (4, 61), (3, 50), (8, 200), (64, 64 * 64 + 3)])
def test_random_ops_match_flat_set(width, n_bits):
    rng = np.random.default_rng(width * 1000 + n_bits)
    hb = O.HierBitmap(n_bits, width=width)
    flat = np.zeros(n_bits, dtype=bool)
    for _ in range(600 if n_bits < 1000 else 300):
        op = rng.integers(0, 4)
        pos = int(rng.integers(0, n_bits))
        if op == 0:
            ok, _ = hb.try_set(pos)
            assert ok == (not flat[pos])
            flat[pos] = True
        elif op == 1:
            ok, _ = hb.try_clear(pos)
            assert ok == bool(flat[pos])
            flat[pos] = False
        elif op == 2:
            i = hb.try_find_set()
            if flat.any():
                assert i is not None and flat[i]
            else:
                assert i is None
        else:
            i = hb.clear_any()
            if i is None:
                assert not flat.any()
            else:
                assert flat[i]
                flat[i] = False
    assert hb.consistent()
    for lv in range(hb.levels):
        assert np.array_equal(hb.level(lv), _nested_from_flat(flat, width, lv)) if n_bits < 1000 else True
    assert np.array_equal(hb.level(0).astype(bool), flat)


def test_levels_until_one_container():
    # A nested bitmap exists iff the level has more bits than one container.
    assert O.HierBitmap(64, 64).levels == 1
    assert O.HierBitmap(65, 64).levels == 2
    assert O.HierBitmap(64 * 64, 64).levels == 2
    assert O.HierBitmap(64 * 64 + 1, 64).levels == 3
    hb = O.HierBitmap(64 ** 3 + 5, 64)
    assert hb.levels == 4
    assert [hb.level_bits(l) for l in range(4)] == [64 ** 3 + 5, 64 * 64 + 1, 65, 2]


def test_cascade_on_all_set_bitmap():
    # An all-set bitmap: clearing a whole container clears exactly one nested bit.
    hb = O.HierBitmap(32, width=4, all_set=True)
    assert hb.consistent()
    for b in (16, 17, 19):
        ok, tr = hb.try_clear(b)
        assert ok and tr == [(0, b)]
    ok, tr = hb.try_clear(18)
    assert ok and tr == [(0, 18), (1, 4)]
    ok, tr = hb.try_set(18)
    assert ok and tr == [(0, 18), (1, 4)]
    assert hb.consistent()
