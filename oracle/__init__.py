"""Oracle for the DynaSOAr hot path: Python access to ``liboracle.so``.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It is independent of
the CUDA library: nothing here loads, calls or shares code with it.

Each function follows the C++ source that states its definition; see
``oracle.h`` for the list and the paper passages they follow.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        u64, i64, i32, dbl = C.c_uint64, C.c_int64, C.c_int, C.c_double
        vp = C.c_void_p
        L.orc_mix64.restype = u64
        L.orc_mix64.argtypes = [u64]
        L.orc_splitmix_at.restype = u64
        L.orc_splitmix_at.argtypes = [u64, u64]
        L.orc_rand.restype = u64
        L.orc_rand.argtypes = [u64, u64, u64, u64]
        L.orc_obj_hash.restype = u64
        L.orc_obj_hash.argtypes = [C.c_uint32, vp, i32]

        L.orc_hb_create.restype = vp
        L.orc_hb_create.argtypes = [u64, i32, i32]
        L.orc_hb_destroy.argtypes = [vp]
        L.orc_hb_levels.restype = i32
        L.orc_hb_levels.argtypes = [vp]
        L.orc_hb_level_bits.restype = u64
        L.orc_hb_level_bits.argtypes = [vp, i32]
        L.orc_hb_get.restype = i32
        L.orc_hb_get.argtypes = [vp, i32, u64]
        L.orc_hb_try_clear.restype = i32
        L.orc_hb_try_clear.argtypes = [vp, u64, vp, vp]
        L.orc_hb_try_set.restype = i32
        L.orc_hb_try_set.argtypes = [vp, u64, vp, vp]
        L.orc_hb_try_find_set.restype = i64
        L.orc_hb_try_find_set.argtypes = [vp]
        L.orc_hb_clear_any.restype = i64
        L.orc_hb_clear_any.argtypes = [vp]
        L.orc_hb_consistent.restype = i32
        L.orc_hb_consistent.argtypes = [vp]

        L.orc_check_heap.restype = C.c_uint32
        L.orc_check_heap.argtypes = [u64, i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, vp]

        L.orc_gol_create.restype = vp
        L.orc_gol_create.argtypes = [i32, i32, vp]
        L.orc_gol_destroy.argtypes = [vp]
        L.orc_gol_step.argtypes = [vp, i32]
        L.orc_gol_alive_count.restype = i64
        L.orc_gol_alive_count.argtypes = [vp]
        L.orc_gol_hash.argtypes = [vp, vp, vp]
        L.orc_gol_dump.restype = i64
        L.orc_gol_dump.argtypes = [vp, vp, vp, i64]

        L.orc_wator_create.restype = vp
        L.orc_wator_create.argtypes = [vp, vp]
        L.orc_wator_destroy.argtypes = [vp]
        L.orc_wator_step.argtypes = [vp, i32, vp]
        L.orc_wator_counts.argtypes = [vp, vp, vp]
        L.orc_wator_hash.argtypes = [vp, vp, vp]
        L.orc_wator_dump.restype = i32
        L.orc_wator_dump.argtypes = [vp, vp, i64, vp, i64]
        L.orc_wator_grid.argtypes = [vp, vp]

        L.orc_set_threads.argtypes = [i32]
        L.orc_nbody_create.restype = vp
        L.orc_nbody_create.argtypes = [vp, vp, i64]
        L.orc_nbody_destroy.argtypes = [vp]
        L.orc_nbody_step.restype = i64
        L.orc_nbody_step.argtypes = [vp, i32, vp, i64, dbl, vp]
        L.orc_nbody_count.restype = i64
        L.orc_nbody_count.argtypes = [vp]
        L.orc_nbody_dump.restype = i64
        L.orc_nbody_dump.argtypes = [vp, vp, i64]

        L.orc_traffic_create.restype = vp
        L.orc_traffic_create.argtypes = [vp, vp]
        L.orc_traffic_destroy.argtypes = [vp]
        L.orc_traffic_step.argtypes = [vp, i32, vp]
        L.orc_traffic_count.restype = i64
        L.orc_traffic_count.argtypes = [vp]
        L.orc_traffic_hash.argtypes = [vp, vp, vp]
        L.orc_traffic_dump.restype = i64
        L.orc_traffic_dump.argtypes = [vp, vp, i64, vp]

        L.orc_sugarscape_create.restype = vp
        L.orc_sugarscape_create.argtypes = [vp, vp, vp, i64]
        L.orc_sugarscape_destroy.argtypes = [vp]
        L.orc_sugarscape_step.argtypes = [vp, i32, vp]
        L.orc_sugarscape_count.restype = i64
        L.orc_sugarscape_count.argtypes = [vp]
        L.orc_sugarscape_hash.restype = u64
        L.orc_sugarscape_hash.argtypes = [vp]
        L.orc_sugarscape_dump.restype = i64
        L.orc_sugarscape_dump.argtypes = [vp, vp, i64, vp]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


# ---- counter-based generator and hash ---------------------------------------
def mix64(z):
    return lib().orc_mix64(z & 0xFFFFFFFFFFFFFFFF)


def splitmix_at(s, n):
    return lib().orc_splitmix_at(s & 0xFFFFFFFFFFFFFFFF, n)


def rand(seed, stream, step, cell):
    return lib().orc_rand(seed, stream, step, cell)


def obj_hash(type_id, words):
    w = np.ascontiguousarray(np.asarray(words, dtype=np.int64).astype(np.uint32))
    return lib().orc_obj_hash(type_id, _ptr(w), len(w))


# ---- hierarchical bitmap model ----------------------------------------------
class HierBitmap:
    """Sequential hierarchical bitmap with a container width parameter (Section 3)."""

    def __init__(self, n_bits, width=64, all_set=False):
        self._h = lib().orc_hb_create(n_bits, width, 1 if all_set else 0)
        if not self._h:
            raise ValueError("width must lie in [2, 64]")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_hb_destroy(self._h)
            self._h = None

    @property
    def levels(self):
        return lib().orc_hb_levels(self._h)

    def level_bits(self, level):
        return lib().orc_hb_level_bits(self._h, level)

    def get(self, level, pos):
        return bool(lib().orc_hb_get(self._h, level, pos))

    def level(self, level):
        return np.array([self.get(level, i) for i in range(self.level_bits(level))], dtype=np.uint8)

    def _traced(self, fn, pos):
        trace = np.zeros(2 * 64, dtype=np.int64)
        n = C.c_int(0)
        ok = fn(self._h, pos, _ptr(trace), C.byref(n))
        return bool(ok), [(int(trace[2 * i]), int(trace[2 * i + 1])) for i in range(n.value)]

    def try_clear(self, pos):
        return self._traced(lib().orc_hb_try_clear, pos)

    def try_set(self, pos):
        return self._traced(lib().orc_hb_try_set, pos)

    def try_find_set(self):
        r = lib().orc_hb_try_find_set(self._h)
        return None if r < 0 else r

    def clear_any(self):
        r = lib().orc_hb_clear_any(self._h)
        return None if r < 0 else r

    def consistent(self):
        return bool(lib().orc_hb_consistent(self._h))


# ---- heap invariants ---------------------------------------------------------
INV_CONTAINER = 1
INV_ONE_STATE = 2
INV_ALLOCATED = 4
INV_ACTIVE = 8
INV_RANGE = 16
INV_STRUCTURE = 32


def check_heap(M, capacity, obj_free, block_type, free_bm, alloc_bm, active_bm, words_per_level, width=64):
    """Check block-state invariants of a heap snapshot; returns (violations, live per type).

    free_bm: u64[total_words]; alloc_bm / active_bm: u64[n_types, total_words],
    each the concatenation of a bitmap's levels (level 0 first), every word
    holding `width` bits (64, 32 or 16).
    """
    n_types = len(capacity)
    cap = np.ascontiguousarray(capacity, dtype=np.uint32)
    of = np.ascontiguousarray(obj_free, dtype=np.uint64)
    bt = np.ascontiguousarray(block_type, dtype=np.uint8)
    fb = np.ascontiguousarray(free_bm, dtype=np.uint64)
    ab = np.ascontiguousarray(alloc_bm, dtype=np.uint64)
    cb = np.ascontiguousarray(active_bm, dtype=np.uint64)
    wpl = np.ascontiguousarray(words_per_level, dtype=np.uint64)
    live = np.zeros(n_types, dtype=np.uint64)
    bad = lib().orc_check_heap(M, n_types, _ptr(cap), _ptr(of), _ptr(bt), _ptr(fb), _ptr(ab), _ptr(cb),
                               _ptr(wpl), len(wpl), int(width), _ptr(live))
    return int(bad), live.astype(np.int64)


# ---- applications ------------------------------------------------------------
class Gol:
    """Game of life (B3/S23) as three do-alls per generation over Cell and Alive."""

    def __init__(self, W, H, alive0):
        a = np.ascontiguousarray(alive0, dtype=np.uint8).reshape(-1)
        assert a.size == W * H
        self.W, self.H = W, H
        self._h = lib().orc_gol_create(W, H, _ptr(a))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_gol_destroy(self._h)
            self._h = None

    def step(self, n=1):
        lib().orc_gol_step(self._h, n)

    def alive_count(self):
        return lib().orc_gol_alive_count(self._h)

    def hash(self):
        a, b = C.c_uint64(0), C.c_uint64(0)
        lib().orc_gol_hash(self._h, C.byref(a), C.byref(b))
        return a.value, b.value

    def dump(self):
        n = self.W * self.H
        cells = np.zeros((n, 3), dtype=np.int32)
        alive = np.zeros((n, 2), dtype=np.int32)
        k = lib().orc_gol_dump(self._h, _ptr(cells), _ptr(alive), n)
        return cells, alive[:k]

    def grid(self):
        cells, _ = self.dump()
        return cells[:, 0].reshape(self.H, self.W).astype(np.uint8)


class _WatorParams(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("seed", C.c_uint64), ("fish_breed", C.c_int32),
                ("shark_breed", C.c_int32), ("shark_energy0", C.c_int32), ("shark_gain", C.c_int32)]


class Wator:
    """Wa-Tor predator-prey as five do-alls per step (F1, F2, S0, S1, S2)."""

    def __init__(self, W, H, kind0, seed, fish_breed=3, shark_breed=10, shark_energy0=5, shark_gain=3):
        k = np.ascontiguousarray(kind0, dtype=np.uint8).reshape(-1)
        assert k.size == W * H
        self.W, self.H = W, H
        self._p = _WatorParams(W, H, seed, fish_breed, shark_breed, shark_energy0, shark_gain)
        self._h = lib().orc_wator_create(C.byref(self._p), _ptr(k))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_wator_destroy(self._h)
            self._h = None

    def step(self, n=1):
        """Advance n steps; returns int64[n, 6] events (fish births, eaten, shark
        births, starved, fish moves, shark moves)."""
        ev = np.zeros((max(n, 1), 6), dtype=np.int64)
        lib().orc_wator_step(self._h, n, _ptr(ev))
        return ev[:n]

    def counts(self):
        a, b = C.c_int64(0), C.c_int64(0)
        lib().orc_wator_counts(self._h, C.byref(a), C.byref(b))
        return a.value, b.value

    def hash(self):
        a, b = C.c_uint64(0), C.c_uint64(0)
        lib().orc_wator_hash(self._h, C.byref(a), C.byref(b))
        return a.value, b.value

    def dump(self):
        nf, ns = self.counts()
        f = np.zeros((max(nf, 1), 3), dtype=np.int32)
        s = np.zeros((max(ns, 1), 4), dtype=np.int32)
        rc = lib().orc_wator_dump(self._h, _ptr(f), nf, _ptr(s), ns)
        assert rc == 0
        return f[:nf], s[:ns]

    def grid(self):
        g = np.zeros(self.W * self.H, dtype=np.uint8)
        lib().orc_wator_grid(self._h, _ptr(g))
        return g.reshape(self.H, self.W)


def set_threads(n):
    """Threads for the per-body rows of the n-body oracle (results do not depend on it)."""
    lib().orc_set_threads(int(n))


class _NBodyParams(C.Structure):
    _fields_ = [("G", C.c_double), ("eps", C.c_double), ("dt", C.c_double), ("r_merge", C.c_double)]


class NBody:
    """N-body with merging collisions in FP64."""

    def __init__(self, bodies, G=1.0, eps=1e-3, dt=1e-4, r_merge=2e-3):
        b = np.ascontiguousarray(bodies, dtype=np.float64)
        assert b.ndim == 2 and b.shape[1] == 7
        self.n0 = b.shape[0]
        self._p = _NBodyParams(G, eps, dt, r_merge)
        self._h = lib().orc_nbody_create(C.byref(self._p), _ptr(b), b.shape[0])

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_nbody_destroy(self._h)
            self._h = None

    def step(self, n=1, margin=0.0, max_merges=1 << 16):
        """Advance n steps; returns (merges int64[k, 3] of (step, survivor, absorbed), marginal pairs)."""
        mg = np.zeros((max_merges, 3), dtype=np.int64)
        marg = C.c_int64(0)
        k = lib().orc_nbody_step(self._h, n, _ptr(mg), max_merges, margin, C.byref(marg))
        return mg[:min(k, max_merges)], marg.value

    def count(self):
        return lib().orc_nbody_count(self._h)

    def dump(self):
        """float64[n, 8] rows (id, x, y, z, vx, vy, vz, m) sorted by id."""
        out = np.zeros((max(self.n0, 1), 8), dtype=np.float64)
        k = lib().orc_nbody_dump(self._h, _ptr(out), self.n0)
        return out[:k]


class _TrafficParams(C.Structure):
    _fields_ = [("R", C.c_int32), ("L", C.c_int32), ("vmax", C.c_int32), ("v_entry", C.c_int32),
                ("periodic", C.c_int32), ("pad_", C.c_int32), ("seed", C.c_uint64), ("p_thr", C.c_uint64),
                ("a_thr", C.c_uint64)]


def prob_threshold(p):
    """floor(p * 2^32): a 32-bit draw u is below probability p iff u < this."""
    assert 0.0 <= p <= 1.0
    return int(np.floor(p * 4294967296.0))


class Traffic:
    """Nagel-Schreckenberg traffic on R single-lane roads of L cells as two
    do-alls per step (Car, then Source on open roads); rules in
    orc_traffic.cpp."""

    def __init__(self, R, L, v0, seed, vmax=5, p=0.25, alpha=0.5, v_entry=None, periodic=False):
        v = np.ascontiguousarray(v0, dtype=np.int8).reshape(-1)
        assert v.size == R * L
        self.R, self.L, self.periodic = R, L, bool(periodic)
        self._p = _TrafficParams(R, L, vmax, vmax if v_entry is None else v_entry, int(bool(periodic)), 0, seed,
                                 prob_threshold(p), prob_threshold(alpha))
        self._h = lib().orc_traffic_create(C.byref(self._p), _ptr(v))
        assert self._h, "invalid traffic parameters"

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_traffic_destroy(self._h)
            self._h = None

    def step(self, n=1):
        """Advance n steps; returns int64[n, 4] events (entered, left, moved,
        velocity sum)."""
        ev = np.zeros((max(n, 1), 4), dtype=np.int64)
        lib().orc_traffic_step(self._h, n, _ptr(ev))
        return ev[:n]

    def count(self):
        return int(lib().orc_traffic_count(self._h))

    def hash(self):
        a, b = C.c_uint64(0), C.c_uint64(0)
        lib().orc_traffic_hash(self._h, C.byref(a), C.byref(b))
        return a.value, b.value

    def dump(self):
        """(cars int32[n, 3] (road, x, v) sorted, sources int32[R or 0, 3])."""
        n = self.count()
        cars = np.zeros((max(n, 1), 3), dtype=np.int32)
        src = np.zeros((self.R, 3), dtype=np.int32)
        assert lib().orc_traffic_dump(self._h, _ptr(cars), n, _ptr(src)) == n
        return cars[:n], (src[:0] if self.periodic else src)


class _SugarParams(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("seed", C.c_uint64), ("alpha", C.c_int32),
                ("endow_lo", C.c_int32), ("endow_hi", C.c_int32), ("metab_lo", C.c_int32), ("metab_hi", C.c_int32),
                ("vision_lo", C.c_int32), ("vision_hi", C.c_int32), ("age_lo", C.c_int32), ("age_hi", C.c_int32)]


class Sugarscape:
    """Sugarscape (Epstein-Axtell rules M, G_alpha, R) as four do-alls per
    step; rules in orc_sugarscape.cpp.

    cap: uint8[H, W] capacities; agents0: int32[n, 7] (x, y, sugar,
    metabolism, vision, age, max_age)."""

    def __init__(self, W, H, cap, agents0, seed, alpha=1, endow=(5, 25), metab=(1, 4), vision=(1, 6),
                 max_age=(60, 100)):
        c = np.ascontiguousarray(cap, dtype=np.uint8).reshape(-1)
        a = np.ascontiguousarray(agents0, dtype=np.int32).reshape(-1, 7)
        assert c.size == W * H
        self.W, self.H = W, H
        self._p = _SugarParams(W, H, seed, alpha, endow[0], endow[1], metab[0], metab[1], vision[0], vision[1],
                               max_age[0], max_age[1])
        self._h = lib().orc_sugarscape_create(C.byref(self._p), _ptr(c), _ptr(a), len(a))
        assert self._h, "invalid sugarscape parameters or agents"

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_sugarscape_destroy(self._h)
            self._h = None

    def step(self, n=1):
        """Advance n steps; returns int64[n, 5] events (moves, starved, aged,
        replacements placed elsewhere, sugar harvested)."""
        ev = np.zeros((max(n, 1), 5), dtype=np.int64)
        lib().orc_sugarscape_step(self._h, n, _ptr(ev))
        return ev[:n]

    def count(self):
        return int(lib().orc_sugarscape_count(self._h))

    def hash(self):
        return int(lib().orc_sugarscape_hash(self._h))

    def dump(self):
        """(agents int32[n, 8] sorted, sugar int32[H, W])."""
        n = self.count()
        a = np.zeros((max(n, 1), 8), dtype=np.int32)
        sg = np.zeros(self.W * self.H, dtype=np.int32)
        assert lib().orc_sugarscape_dump(self._h, _ptr(a), n, _ptr(sg)) == n
        return a[:n], sg.reshape(self.H, self.W)
