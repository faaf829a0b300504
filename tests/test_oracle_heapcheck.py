"""Oracle pins: the heap invariant checker accepts consistent heaps and flags each planted violation."""
import numpy as np
import pytest

import oracle as O


def _levels(M, width=64):
    bits = [M]
    while bits[-1] > width:
        bits.append(-(-bits[-1] // width))
    return bits, [-(-b // width) for b in bits]


def _bitmap(flags, M, width=64):
    """Hierarchical bitmap words (levels concatenated) for per-position flags:
    position p of a level is bit p % width of word p // width."""
    bits, words = _levels(M, width)
    out = []
    cur = np.asarray(flags, dtype=bool)
    for l, w in enumerate(words):
        padded = np.zeros(w * width, dtype=bool)
        padded[:len(cur)] = cur
        full = np.zeros((w, 64), dtype=bool)
        full[:, :width] = padded.reshape(w, width)
        ws = np.packbits(full[:, ::-1], axis=1).view(">u8").reshape(w).astype(np.uint64)
        out.append(ws)
        cur = padded.reshape(w, width).any(axis=1)
    return np.concatenate(out), np.array(words, dtype=np.uint64)


def _heap(seed=0, M=300, caps=(64, 40), width=64):
    rng = np.random.default_rng(seed)
    T = len(caps)
    state = rng.integers(-1, T, M)  # -1 free
    obj_free = np.zeros(M, dtype=np.uint64)
    btype = np.full(M, 0xFF, dtype=np.uint8)
    live = np.zeros(T, dtype=np.int64)
    for b in range(M):
        t = state[b]
        if t < 0:
            continue
        c = caps[t]
        occ = rng.random(c) < rng.choice([0.3, 1.0])
        if not occ.any():
            occ[rng.integers(0, c)] = True
        live[t] += occ.sum()
        fr = 0
        for s in range(c):
            if not occ[s]:
                fr |= 1 << s
        obj_free[b] = np.uint64(fr)
        btype[b] = t
    free_bm, wpl = _bitmap(state < 0, M, width)
    alloc = np.stack([_bitmap(state == t, M, width)[0] for t in range(T)])
    active = np.stack([_bitmap((state == t) & (obj_free != 0), M, width)[0] for t in range(T)])
    return dict(M=M, capacity=np.array(caps), obj_free=obj_free, block_type=btype, free_bm=free_bm,
                alloc_bm=alloc, active_bm=active, words_per_level=wpl, width=width), live


@pytest.mark.parametrize("seed,M", [(0, 300), (1, 64), (2, 5000), (3, 64 * 64 + 7)])
@pytest.mark.parametrize("width", [64, 32, 16])
def test_consistent_heap_passes(seed, M, width):
    h, live = _heap(seed, M, width=width)
    bad, got = O.check_heap(**h)
    assert bad == 0
    assert np.array_equal(got, live)


def test_level_counts_follow_the_width():
    # 5000 blocks: 64-bit containers give 79 + 2 + 1 words, 16-bit ones
    # 313 + 20 + 2 + 1
    assert _levels(5000, 64)[1] == [79, 2, 1]
    assert _levels(5000, 16)[1] == [313, 20, 2, 1]
    h, _ = _heap(2, 5000, width=16)
    assert O.check_heap(**dict(h, width=64))[0] & O.INV_STRUCTURE  # read with the wrong width


@pytest.mark.parametrize("width", [32, 16])
def test_narrow_width_flags_bits_beyond_the_width_and_nesting(width):
    h, _ = _heap(7, 3000, width=width)
    g = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in h.items()}
    g["free_bm"][0] |= np.uint64(1) << np.uint64(width)  # a bit past the container width
    assert O.check_heap(**g)[0] & O.INV_RANGE
    g = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in h.items()}
    n0 = int(g["words_per_level"][0])
    g["alloc_bm"][1][n0] ^= np.uint64(1 << 2)  # level-1 bit out of step with its container
    assert O.check_heap(**g)[0] & O.INV_CONTAINER


def test_flags_each_planted_violation():
    h, _ = _heap(5, 300)
    full_block = int(np.nonzero((h["block_type"] == 0) & (h["obj_free"] == 0))[0][0])
    free_block = int(np.nonzero(h["block_type"] == 0xFF)[0][0])
    typed_block = int(np.nonzero(h["block_type"] == 1)[0][0])

    def plant(fn, bit):
        g = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in h.items()}
        fn(g)
        bad, _ = O.check_heap(**g)
        assert bad & bit, (bad, bit)

    # I1: a nested bit out of step with its container
    def nested(g):
        n0 = int(g["words_per_level"][0])
        g["free_bm"][n0] ^= np.uint64(1 << 3)
    plant(nested, O.INV_CONTAINER)

    # I5: a free block also allocated
    def two_states(g):
        g["free_bm"][free_block // 64] &= ~np.uint64(0)  # unchanged
        g["alloc_bm"][0][free_block // 64] |= np.uint64(1 << (free_block % 64))
    plant(two_states, O.INV_ONE_STATE)

    # I3: allocated[1] bit on a block whose type byte says 0
    def wrong_type(g):
        g["block_type"][typed_block] = 0
    plant(wrong_type, O.INV_ALLOCATED)

    # I3: an allocated block with no object
    def empty_alloc(g):
        g["obj_free"][typed_block] = np.uint64((1 << 40) - 1)
    plant(empty_alloc, O.INV_ALLOCATED)

    # I4: a full block marked active
    def full_active(g):
        g["active_bm"][0][full_block // 64] |= np.uint64(1 << (full_block % 64))
    plant(full_active, O.INV_ACTIVE)

    # range: a free-slot bit beyond the type's capacity
    def beyond_cap(g):
        g["obj_free"][typed_block] |= np.uint64(1 << 50)
    plant(beyond_cap, O.INV_RANGE)

    # structure: wrong level sizes
    def structure(g):
        g["words_per_level"] = g["words_per_level"][:1]
    plant(structure, O.INV_STRUCTURE)


@pytest.mark.parametrize("width", [64, 32, 16])
def test_expected_stats_counts_block_states(width):
    # the block and object counts the GPU statistics are checked against,
    # on a synthetic consistent heap whose free blocks partly keep the type
    # byte of their last use (a reclaimed block: type T, no free slot, free)
    from helpers import expected_stats
    M, caps = 64 * width + 333, (64, 40)
    h, live = _heap(5, M, caps=caps, width=width)
    rng = np.random.default_rng(9)
    free = h["block_type"] == 0xFF
    reused = free & (rng.random(M) < 0.5)
    h["block_type"][reused] = rng.integers(0, 2, int(reused.sum()))
    st = expected_stats(h)
    assert st["free_blocks"] == int(free.sum())
    for t, c in enumerate(caps):
        mine = (h["block_type"] == t) & ~free
        assert st["allocated_blocks"][t] == int(mine.sum())
        assert st["active_blocks"][t] == int((mine & (h["obj_free"] != 0)).sum())
        assert st["live_objects"][t] == int(live[t])
