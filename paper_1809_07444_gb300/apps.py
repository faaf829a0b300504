"""Python binding of the SMMO applications (include/dsr_apps.h): argument marshalling only."""
import ctypes as C
import math

import numpy as np
import torch

from . import _lib as L
from .heap import Heap, _stream_ptr, heap_bytes_for_blocks

GOL_TYPES = [[4, 4, 4], [4, 4]]          # Cell {alive, count, idx}, Alive {x, y}
WATOR_TYPES = [[4, 4, 4], [4, 4, 4, 4]]  # Fish {x, y, timer}, Shark {x, y, timer, energy}
TRAFFIC_TYPES = [[4, 4, 4], [4, 4, 4]]   # Car {road, x, v}, Source {road, entered, blocked}
SUGAR_TYPES = [[4] * 8]                  # Agent {x, y, sugar, metabolism, vision, age, max_age, dead}


def _sorted_rows(a):
    if len(a) == 0:
        return a.reshape(0, a.shape[1] if a.ndim == 2 else 0)
    idx = np.lexsort(a.T[::-1])
    return a[idx]


def _blocks_for(cells, caps, slack=2.0, tuning=None):
    """Blocks for `cells` objects of each type with the given capacities at
    cap_min 64 (scaled down with a smaller cap_min), with slack."""
    scale = int((tuning or {}).get("cap_min") or 64) / 64.0
    return int(slack * sum(math.ceil(cells / max(1, int(c * scale))) for c in caps)) + 256


class Gol:
    """Game of life (B3/S23) on a W x H torus, driven through libdsr."""

    def __init__(self, W, H, alive0, heap_bytes=None, tuning=None, stream=None):
        self.lib = L.load()
        self.W, self.H = W, H
        if heap_bytes is None:
            heap_bytes = heap_bytes_for_blocks(GOL_TYPES, _blocks_for(W * H, [42, 64], tuning=tuning), tuning)
        self.heap = Heap(GOL_TYPES, heap_bytes, names=["Cell", "Alive"], tuning=tuning, stream=stream)
        ws = C.c_size_t(0)
        L.check(self.lib.dsr_gol_workspace_bytes(W, H, C.byref(ws)), "dsr_gol_workspace_bytes")
        self.workspace = torch.empty(ws.value, dtype=torch.uint8, device="cuda")
        a0 = torch.as_tensor(np.ascontiguousarray(alive0, dtype=np.uint8).reshape(-1)).cuda()
        h = C.c_void_p()
        L.check(self.lib.dsr_gol_create(self.heap.handle, W, H, C.c_void_p(a0.data_ptr()),
                                        C.c_void_p(self.workspace.data_ptr()), _stream_ptr(stream), C.byref(h)),
                "dsr_gol_create")
        self.handle = h
        self._a0 = a0

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.dsr_gol_destroy(self.handle)
            self.handle = None

    def step(self, n=1, stream=None):
        L.check(self.lib.dsr_gol_step(self.handle, n, _stream_ptr(stream)), "dsr_gol_step")

    def method_args(self):
        return L.GolArgs(C.c_void_p(self.workspace.data_ptr()), self.W, self.H)

    def dump(self):
        """(cells int32[W*H, 3] in idx order, alive int32[k, 2] sorted)."""
        cf, _ = self.heap.dump(0)
        af, _ = self.heap.dump(1)
        cells = cf.view(np.int32)
        cells = cells[np.argsort(cells[:, 2], kind="stable")]
        return cells, _sorted_rows(af.view(np.int32))

    def hash(self):
        return self.heap.hash(0), self.heap.hash(1)


class Wator:
    """Wa-Tor predator-prey on a W x H torus, driven through libdsr."""

    def __init__(self, W, H, kind0, seed, fish_breed=3, shark_breed=10, shark_energy0=5, shark_gain=3,
                 heap_bytes=None, tuning=None, stream=None):
        self.lib = L.load()
        self.W, self.H = W, H
        if heap_bytes is None:
            heap_bytes = heap_bytes_for_blocks(WATOR_TYPES, _blocks_for(W * H, [48], tuning=tuning), tuning)
        self.heap = Heap(WATOR_TYPES, heap_bytes, names=["Fish", "Shark"], tuning=tuning, stream=stream)
        ws = C.c_size_t(0)
        L.check(self.lib.dsr_wator_workspace_bytes(self.heap.handle, W, H, C.byref(ws)), "dsr_wator_workspace_bytes")
        self.workspace = torch.empty(ws.value, dtype=torch.uint8, device="cuda")
        k0 = torch.as_tensor(np.ascontiguousarray(kind0, dtype=np.uint8).reshape(-1)).cuda()
        self.params = L.WatorParams(W, H, seed, fish_breed, shark_breed, shark_energy0, shark_gain)
        h = C.c_void_p()
        L.check(self.lib.dsr_wator_create(self.heap.handle, C.byref(self.params), C.c_void_p(k0.data_ptr()),
                                          C.c_void_p(self.workspace.data_ptr()), _stream_ptr(stream),
                                          C.byref(h)), "dsr_wator_create")
        self.handle = h
        self._k0 = k0

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.dsr_wator_destroy(self.handle)
            self.handle = None

    def checkpoint(self):
        """Host copies of the heap arena and the workspace, with what a
        restore needs (see dsr_wator_attach)."""
        torch.cuda.synchronize()
        return {"W": self.W, "H": self.H, "params": bytes(self.params), "tuning": self.heap.tuning,
                "arena": self.heap.arena.cpu(), "workspace": self.workspace.cpu()}

    @classmethod
    def restore(cls, ck, stream=None):
        """A Wator that continues from a checkpoint, bit for bit."""
        w = cls.__new__(cls)
        w.lib = L.load()
        w.W, w.H = ck["W"], ck["H"]
        w.heap = Heap(WATOR_TYPES, ck["arena"].numel(), names=["Fish", "Shark"], tuning=ck["tuning"], stream=stream)
        torch.cuda.synchronize()  # the creation's reset has run
        w.heap.arena.copy_(ck["arena"])
        w.workspace = ck["workspace"].cuda()
        w.params = L.WatorParams.from_buffer_copy(ck["params"])
        h = C.c_void_p()
        L.check(w.lib.dsr_wator_attach(w.heap.handle, C.byref(w.params), C.c_void_p(w.workspace.data_ptr()),
                                       C.byref(h)), "dsr_wator_attach")
        w.handle = h
        return w

    def step(self, n=1, stream=None):
        L.check(self.lib.dsr_wator_step(self.handle, n, _stream_ptr(stream)), "dsr_wator_step")

    def counts(self):
        st = self.heap.stats()
        return st["live_objects"][0], st["live_objects"][1]

    PHASES = ("F1", "F2", "S0", "S1", "S2")

    def phase_timing(self, max_steps):
        """Record CUDA events around every scan and method kernel of the next
        max_steps steps (0 turns it off)."""
        L.check(self.lib.dsr_wator_phase_timing(self.handle, int(max_steps)), "dsr_wator_phase_timing")

    def phase_select(self, phase):
        """Time only the method kernel of one phase (its index in PHASES), or
        every scan and method kernel with None; starts a new window."""
        L.check(self.lib.dsr_wator_phase_select(self.handle, -1 if phase is None else int(phase)),
                "dsr_wator_phase_select")

    def phase_times(self):
        """({phase: method-kernel ms}, {phase: scan ms}, steps) summed over the
        steps recorded since the last call."""
        out = (C.c_double * 10)()
        n = C.c_int(0)
        L.check(self.lib.dsr_wator_phase_times(self.handle, out, C.byref(n)), "dsr_wator_phase_times")
        return ({p: out[i] for i, p in enumerate(self.PHASES)}, {p: out[5 + i] for i, p in enumerate(self.PHASES)},
                n.value)

    def dump(self):
        """(fish int32[n, 3] sorted, sharks int32[m, 4] sorted)."""
        f, _ = self.heap.dump(0)
        s, _ = self.heap.dump(1)
        return _sorted_rows(f.view(np.int32)), _sorted_rows(s.view(np.int32))

    def hash(self):
        return self.heap.hash(0), self.heap.hash(1)

    def grid(self):
        out = torch.empty(self.W * self.H, dtype=torch.uint8, device="cuda")
        L.check(self.lib.dsr_wator_kinds(self.handle, C.c_void_p(out.data_ptr()), _stream_ptr()), "dsr_wator_kinds")
        return out.cpu().numpy().reshape(self.H, self.W)


class WatorBitmap:
    """Wa-tor on the BitmapAlloc comparator heap (same rules as Wator);
    capacity per type defaults to one object per cell."""

    def __init__(self, W, H, kind0, seed, capacity=None, fish_breed=3, shark_breed=10, shark_energy0=5,
                 shark_gain=3, stream=None):
        from .heap import BitmapHeap
        self.lib = L.load()
        self.W, self.H = W, H
        n = -(-(W * H) // 64) * 64
        self.heap = BitmapHeap(WATOR_TYPES, capacity or [n, n], stream=stream)
        ws = C.c_size_t(0)
        L.check(self.lib.dsr_wator_bm_workspace_bytes(self.heap.handle, W, H, C.byref(ws)),
                "dsr_wator_bm_workspace_bytes")
        self.workspace = torch.empty(ws.value, dtype=torch.uint8, device="cuda")
        k0 = torch.as_tensor(np.ascontiguousarray(kind0, dtype=np.uint8).reshape(-1)).cuda()
        self.params = L.WatorParams(W, H, seed, fish_breed, shark_breed, shark_energy0, shark_gain)
        h = C.c_void_p()
        L.check(self.lib.dsr_wator_bm_create(self.heap.handle, C.byref(self.params), C.c_void_p(k0.data_ptr()),
                                             C.c_void_p(self.workspace.data_ptr()), _stream_ptr(stream),
                                             C.byref(h)), "dsr_wator_bm_create")
        self.handle = h
        self._k0 = k0

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.dsr_wator_bm_destroy(self.handle)
            self.handle = None

    def step(self, n=1, stream=None):
        L.check(self.lib.dsr_wator_bm_step(self.handle, n, _stream_ptr(stream)), "dsr_wator_bm_step")

    def hash(self):
        return self.heap.hash(0), self.heap.hash(1)

    def counts(self):
        return tuple(self.heap.stats()["live_objects"])


class WatorStatic:
    """Wa-tor without dynamic allocation (per-cell arrays; aos selects the
    layout), the comparator of the allocator-based form."""

    def __init__(self, W, H, kind0, seed, aos=False, fish_breed=3, shark_breed=10, shark_energy0=5, shark_gain=3,
                 stream=None):
        self.lib = L.load()
        self.W, self.H = W, H
        n = C.c_size_t(0)
        L.check(self.lib.dsr_wator_static_bytes(W, H, 1 if aos else 0, C.byref(n)), "dsr_wator_static_bytes")
        self.workspace = torch.empty(n.value, dtype=torch.uint8, device="cuda")
        k0 = torch.as_tensor(np.ascontiguousarray(kind0, dtype=np.uint8).reshape(-1)).cuda()
        self.params = L.WatorParams(W, H, seed, fish_breed, shark_breed, shark_energy0, shark_gain)
        h = C.c_void_p()
        L.check(self.lib.dsr_wator_static_create(C.byref(self.params), C.c_void_p(k0.data_ptr()),
                                                 C.c_void_p(self.workspace.data_ptr()), 1 if aos else 0,
                                                 _stream_ptr(stream), C.byref(h)), "dsr_wator_static_create")
        self.handle = h
        self._k0 = k0

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.dsr_wator_static_destroy(self.handle)
            self.handle = None

    def step(self, n=1, stream=None):
        L.check(self.lib.dsr_wator_static_step(self.handle, n, _stream_ptr(stream)), "dsr_wator_static_step")

    def hash(self):
        out = torch.zeros(2, dtype=torch.int64, device="cuda")
        L.check(self.lib.dsr_wator_static_hash(self.handle, C.c_void_p(out.data_ptr()), _stream_ptr()),
                "dsr_wator_static_hash")
        v = out.cpu().numpy().view(np.uint64)
        return int(v[0]), int(v[1])

    def state(self):
        n = self.W * self.H
        k = torch.empty(n, dtype=torch.uint8, device="cuda")
        t = torch.empty(n, dtype=torch.int32, device="cuda")
        e = torch.empty(n, dtype=torch.int32, device="cuda")
        L.check(self.lib.dsr_wator_static_state(self.handle, C.c_void_p(k.data_ptr()), C.c_void_p(t.data_ptr()),
                                                C.c_void_p(e.data_ptr()), _stream_ptr()), "dsr_wator_static_state")
        return k.cpu().numpy(), t.cpu().numpy(), e.cpu().numpy()

    def dump(self):
        """(fish int32[n, 3] sorted, sharks int32[m, 4] sorted), as Wator.dump."""
        k, t, e = self.state()
        c = np.arange(self.W * self.H)
        x, y = (c % self.W).astype(np.int32), (c // self.W).astype(np.int32)
        f = k == 1
        s = k == 2
        fish = np.stack([x[f], y[f], t[f]], axis=1).astype(np.int32)
        sharks = np.stack([x[s], y[s], t[s], e[s]], axis=1).astype(np.int32)
        return _sorted_rows(fish), _sorted_rows(sharks)

    def grid(self):
        return self.state()[0].reshape(self.H, self.W)

    def visits(self):
        v = C.c_uint64(0)
        L.check(self.lib.dsr_wator_static_visits(self.handle, C.byref(v)), "dsr_wator_static_visits")
        return int(v.value)


def _heap_base(lib, handle):
    """Device address of a heap's arena (its device view starts with the data pointer)."""
    n = lib.dsr_dev_heap_size()
    buf = (C.c_uint8 * n)()
    L.check(lib.dsr_heap_device_view(handle, buf, n), "dsr_heap_device_view")
    data = C.c_uint64.from_buffer(buf, 0).value
    lay = L.Layout()
    L.check(lib.dsr_heap_layout(handle, C.byref(lay)), "dsr_heap_layout")
    return data - lay.off_data


def _group_free_bytes(lib, g):
    """(free bytes, largest free range) of a group's arena."""
    t, l = C.c_size_t(0), C.c_size_t(0)
    L.check(lib.dsr_group_free_bytes(g, C.byref(t), C.byref(l)), "dsr_group_free_bytes")
    return int(t.value), int(l.value)


class WatorBatch:
    """Many wa-tor instances in one arena, stepped together by graph-captured group do-alls."""

    def __init__(self, arena_bytes=None, max_instances=256, tuning=None, stream=None, share=None):
        """A new arena of arena_bytes, or (share=another batch) that batch's
        arena, whose free bytes the two then draw on together."""
        from .heap import _tuning
        self.lib = L.load()
        self.tuning = tuning
        tun = _tuning(tuning)
        h = C.c_void_p()
        if share is None:
            self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device="cuda")
            L.check(self.lib.dsr_wator_batch_create(C.c_void_p(self.arena.data_ptr()), int(arena_bytes), max_instances,
                                                    C.byref(tun) if tun else None, _stream_ptr(stream), C.byref(h)),
                    "dsr_wator_batch_create")
        else:
            self.arena, self._share = share.arena, share
            L.check(self.lib.dsr_wator_batch_create_shared(share.group(), max_instances, C.byref(tun) if tun else None,
                                                           _stream_ptr(stream), C.byref(h)),
                    "dsr_wator_batch_create_shared")
        self.handle = h
        self.inst = {}  # slot -> (W, H, params)
        self._kinds = {}

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.dsr_wator_batch_destroy(self.handle)
            self.handle = None

    @staticmethod
    def blocks_for(W, H, tuning=None):
        return _blocks_for(W * H, [48], tuning=tuning)

    def instance_bytes(self, W, H, n_blocks=None):
        out = C.c_size_t(0)
        L.check(self.lib.dsr_wator_batch_instance_bytes(self.handle, W, H, n_blocks or self.blocks_for(W, H, self.tuning),
                                                        C.byref(out)), "dsr_wator_batch_instance_bytes")
        return int(out.value)

    def add(self, W, H, kind0, seed, fish_breed=3, shark_breed=10, shark_energy0=5, shark_gain=3, n_blocks=None,
            stream=None):
        """Add an instance; returns its slot, or None when the arena has no room."""
        k0 = torch.as_tensor(np.ascontiguousarray(kind0, dtype=np.uint8).reshape(-1)).cuda()
        p = L.WatorParams(W, H, seed, fish_breed, shark_breed, shark_energy0, shark_gain)
        slot = C.c_int(-1)
        rc = self.lib.dsr_wator_batch_add(self.handle, C.byref(p), n_blocks or self.blocks_for(W, H, self.tuning),
                                          C.c_void_p(k0.data_ptr()), _stream_ptr(stream), C.byref(slot))
        if rc == L.E_OOM:
            return None
        L.check(rc, "dsr_wator_batch_add")
        self.inst[slot.value] = (W, H, p)
        return slot.value

    def remove(self, slot):
        torch.cuda.synchronize()
        L.check(self.lib.dsr_wator_batch_remove(self.handle, slot), "dsr_wator_batch_remove")
        del self.inst[slot]

    def step(self, n=1, stream=None):
        L.check(self.lib.dsr_wator_batch_step(self.handle, n, _stream_ptr(stream)), "dsr_wator_batch_step")

    def prepare(self):
        """Capture the step graph now if the set of instances changed."""
        L.check(self.lib.dsr_wator_batch_prepare(self.handle), "dsr_wator_batch_prepare")

    def group(self):
        g = C.c_void_p()
        L.check(self.lib.dsr_wator_batch_group(self.handle, C.byref(g)), "dsr_wator_batch_group")
        return g

    def free_bytes(self):
        return _group_free_bytes(self.lib, self.group())

    def heap(self, slot):
        h = C.c_void_p()
        L.check(self.lib.dsr_wator_batch_heap(self.handle, slot, C.byref(h)), "dsr_wator_batch_heap")
        off = _heap_base(self.lib, h) - self.arena.data_ptr()
        return Heap.view(h, WATOR_TYPES, self.arena[off:], names=["Fish", "Shark"])

    def hash(self, slot):
        hp = self.heap(slot)
        return hp.hash(0), hp.hash(1)

    def dump(self, slot):
        hp = self.heap(slot)
        f, _ = hp.dump(0)
        s, _ = hp.dump(1)
        return _sorted_rows(f.view(np.int32)), _sorted_rows(s.view(np.int32))

    def counts(self, slot):
        st = self.heap(slot).stats()
        return st["live_objects"][0], st["live_objects"][1]

    def grid(self, slot):
        W, H, _ = self.inst[slot]
        out = torch.empty(W * H, dtype=torch.uint8, device="cuda")
        L.check(self.lib.dsr_wator_batch_kinds(self.handle, slot, C.c_void_p(out.data_ptr()), _stream_ptr()),
                "dsr_wator_batch_kinds")
        return out.cpu().numpy().reshape(H, W)

    def free_bytes(self):
        g = C.c_void_p()
        L.check(self.lib.dsr_wator_batch_group(self.handle, C.byref(g)), "dsr_wator_batch_group")
        t, l = C.c_size_t(0), C.c_size_t(0)
        L.check(self.lib.dsr_group_free_bytes(g, C.byref(t), C.byref(l)), "dsr_group_free_bytes")
        return int(t.value), int(l.value)


class GolBatch:
    """Many game-of-life instances in one arena, stepped together by graph-captured group do-alls."""

    def __init__(self, arena_bytes=None, max_instances=256, tuning=None, stream=None, share=None):
        """A new arena of arena_bytes, or (share=another batch) that batch's
        arena, whose free bytes the two then draw on together."""
        from .heap import _tuning
        self.lib = L.load()
        self.tuning = tuning
        tun = _tuning(tuning)
        h = C.c_void_p()
        if share is None:
            self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device="cuda")
            L.check(self.lib.dsr_gol_batch_create(C.c_void_p(self.arena.data_ptr()), int(arena_bytes), max_instances,
                                                  C.byref(tun) if tun else None, _stream_ptr(stream), C.byref(h)),
                    "dsr_gol_batch_create")
        else:
            self.arena, self._share = share.arena, share
            L.check(self.lib.dsr_gol_batch_create_shared(share.group(), max_instances, C.byref(tun) if tun else None,
                                                         _stream_ptr(stream), C.byref(h)),
                    "dsr_gol_batch_create_shared")
        self.handle = h
        self.inst = {}

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.dsr_gol_batch_destroy(self.handle)
            self.handle = None

    @staticmethod
    def blocks_for(W, H, tuning=None):
        return _blocks_for(W * H, [42, 64], tuning=tuning)

    def instance_bytes(self, W, H, n_blocks=None):
        out = C.c_size_t(0)
        L.check(self.lib.dsr_gol_batch_instance_bytes(self.handle, W, H, n_blocks or self.blocks_for(W, H, self.tuning),
                                                      C.byref(out)), "dsr_gol_batch_instance_bytes")
        return int(out.value)

    def add(self, W, H, alive0, n_blocks=None, stream=None):
        """Add an instance; returns its slot, or None when the arena has no room."""
        a0 = torch.as_tensor(np.ascontiguousarray(alive0, dtype=np.uint8).reshape(-1)).cuda()
        slot = C.c_int(-1)
        rc = self.lib.dsr_gol_batch_add(self.handle, W, H, n_blocks or self.blocks_for(W, H, self.tuning),
                                        C.c_void_p(a0.data_ptr()), _stream_ptr(stream), C.byref(slot))
        if rc == L.E_OOM:
            return None
        L.check(rc, "dsr_gol_batch_add")
        self.inst[slot.value] = (W, H)
        return slot.value

    def remove(self, slot):
        torch.cuda.synchronize()
        L.check(self.lib.dsr_gol_batch_remove(self.handle, slot), "dsr_gol_batch_remove")
        del self.inst[slot]

    def step(self, n=1, stream=None):
        L.check(self.lib.dsr_gol_batch_step(self.handle, n, _stream_ptr(stream)), "dsr_gol_batch_step")

    def prepare(self):
        """Capture the generation graph now if the set of instances changed."""
        L.check(self.lib.dsr_gol_batch_prepare(self.handle), "dsr_gol_batch_prepare")

    def group(self):
        g = C.c_void_p()
        L.check(self.lib.dsr_gol_batch_group(self.handle, C.byref(g)), "dsr_gol_batch_group")
        return g

    def free_bytes(self):
        return _group_free_bytes(self.lib, self.group())

    def heap(self, slot):
        h = C.c_void_p()
        L.check(self.lib.dsr_gol_batch_heap(self.handle, slot, C.byref(h)), "dsr_gol_batch_heap")
        off = _heap_base(self.lib, h) - self.arena.data_ptr()
        return Heap.view(h, GOL_TYPES, self.arena[off:], names=["Cell", "Alive"])

    def hash(self, slot):
        hp = self.heap(slot)
        return hp.hash(0), hp.hash(1)

    def free_bytes(self):
        g = C.c_void_p()
        L.check(self.lib.dsr_gol_batch_group(self.handle, C.byref(g)), "dsr_gol_batch_group")
        t, l = C.c_size_t(0), C.c_size_t(0)
        L.check(self.lib.dsr_group_free_bytes(g, C.byref(t), C.byref(l)), "dsr_group_free_bytes")
        return int(t.value), int(l.value)


# Body {id, x, y, z, vx, vy, vz, m, then the low words of x .. m}: each state
# component is an FP32 pair (high word, low word) whose sum is its value
NBODY_TYPES = [[4] * 15]
NBODY_R_NEAR = 0.02  # pairs closer than this are summed in FP64 (see dsr_apps.h)


class NBody:
    """N-body with merging collisions (FP32-pair state, FP64 update and
    merges), driven through libdsr.

    rows: float[n, 7] (x, y, z, vx, vy, vz, m), each value FP32-representable
    (the stored low words start at 0); body i gets id i.
    pairs: "fp32" (FP32 pair forces, FP64 for pairs closer than r_near) or
    "fp64" (every pair in FP64).
    """

    def __init__(self, rows, G=1.0, eps=1e-3, dt=1e-4, r_merge=2e-3, r_near=NBODY_R_NEAR, pairs="fp32",
                 heap_bytes=None, log_cap=1 << 20, tuning=None, stream=None):
        if pairs not in ("fp32", "fp64"):
            raise ValueError("pairs must be 'fp32' or 'fp64'")
        self.lib = L.load()
        rows = np.ascontiguousarray(rows, dtype=np.float32)
        n = rows.shape[0]
        self.n0 = n
        if heap_bytes is None:
            heap_bytes = heap_bytes_for_blocks(NBODY_TYPES, 2 * (-(-n // 64)) + 64, tuning)
        self.heap = Heap(NBODY_TYPES, heap_bytes, names=["Body"], tuning=tuning, stream=stream)
        ws = C.c_size_t(0)
        L.check(self.lib.dsr_nbody_workspace_bytes(self.heap.handle, log_cap, C.byref(ws)), "dsr_nbody_workspace_bytes")
        self.workspace = torch.empty(ws.value, dtype=torch.uint8, device="cuda")
        self._rows = torch.from_numpy(rows).cuda()
        self.params = L.NBodyParams(G, eps, dt, r_merge, r_near,
                                    L.NBODY_PAIRS_FP64 if pairs == "fp64" else L.NBODY_PAIRS_FP32, 0)
        self.log_cap = log_cap
        h = C.c_void_p()
        L.check(self.lib.dsr_nbody_create(self.heap.handle, C.byref(self.params), C.c_void_p(self._rows.data_ptr()),
                                          n, C.c_void_p(self.workspace.data_ptr()), log_cap, _stream_ptr(stream),
                                          C.byref(h)), "dsr_nbody_create")
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.dsr_nbody_destroy(self.handle)
            self.handle = None

    def step(self, n=1, stream=None):
        L.check(self.lib.dsr_nbody_step(self.handle, n, _stream_ptr(stream)), "dsr_nbody_step")

    def dump(self):
        """float64[k, 8] rows (id, x, y, z, vx, vy, vz, m) sorted by id; each
        value is the sum of its stored high and low words."""
        return nbody_rows(self.heap)

    def _ws_word(self, ptr, dtype, count=1):
        torch.cuda.synchronize()
        off = ptr - self.workspace.data_ptr()
        size = np.dtype(dtype).itemsize * count
        return self.workspace[off: off + size].cpu().numpy().view(dtype)

    def merges(self):
        """int64[k, 3] merge log rows (step, survivor id, absorbed id), sorted."""
        lp, cp = C.c_void_p(), C.c_void_p()
        L.check(self.lib.dsr_nbody_merge_log(self.handle, C.byref(lp), C.byref(cp)), "dsr_nbody_merge_log")
        n = int(self._ws_word(cp.value, np.uint64)[0])  # the log and its count live in the workspace
        if n > self.log_cap:
            raise L.DsrError("merge log overflow: %d > %d" % (n, self.log_cap))
        log = self._ws_word(lp.value, np.int32, 3 * n).reshape(n, 3).astype(np.int64)
        return log[np.lexsort(log.T[::-1])] if n else log

    def near_pairs(self):
        """Near pairs (closer than r_near, each counted from both bodies) of the last step."""
        cp = C.c_void_p()
        L.check(self.lib.dsr_nbody_near_pairs(self.handle, C.byref(cp)), "dsr_nbody_near_pairs")
        return int(self._ws_word(cp.value, np.uint32)[0])


def nbody_rows(heap):
    """float64[k, 8] rows (id, x, y, z, vx, vy, vz, m) of the bodies of an
    n-body heap, sorted by id; each value is its high word plus its low word."""
    f, _ = heap.dump(0)
    w = f[:, 1:15].view(np.float32).astype(np.float64)
    out = np.zeros((len(f), 8), dtype=np.float64)
    out[:, 0] = f[:, 0].view(np.int32)
    out[:, 1:] = w[:, 0:7] + w[:, 7:14]
    return out[np.argsort(out[:, 0], kind="stable")]


_LIBMOD = L  # Traffic's road length is named L, after the model


def prob_threshold(p):
    """floor(p * 2^32): a 32-bit draw u counts as below probability p iff u < this."""
    if not 0.0 <= p <= 1.0:
        raise ValueError("probability out of range")
    return int(math.floor(p * 4294967296.0))


class Traffic:
    """Nagel-Schreckenberg traffic on R single-lane roads of L cells, driven
    through libdsr (rules in include/dsr_apps.h).

    v0: int8[R, L], -1 for an empty cell, else the car's initial velocity.
    periodic: ring roads; otherwise open roads with a Source per road that
    admits cars with probability alpha at velocity v_entry (default vmax).
    """

    def __init__(self, R, L, v0, seed, vmax=5, p=0.25, alpha=0.5, v_entry=None, periodic=False,
                 heap_bytes=None, tuning=None, stream=None):
        if np.asarray(v0).size != R * L:
            raise ValueError("v0 must have R * L cells")
        self.lib = _LIBMOD.load()
        self.R, self.L, self.periodic = R, L, bool(periodic)
        self.params = _LIBMOD.TrafficParams(R, L, vmax, vmax if v_entry is None else v_entry, int(bool(periodic)), 0,
                                      seed, prob_threshold(p), prob_threshold(alpha))
        if heap_bytes is None:
            blocks = _blocks_for(R * L, [64], tuning=tuning) + math.ceil(R / 64)
            heap_bytes = heap_bytes_for_blocks(TRAFFIC_TYPES, blocks, tuning)
        self.heap = Heap(TRAFFIC_TYPES, heap_bytes, names=["Car", "Source"], tuning=tuning, stream=stream)
        ws = C.c_size_t(0)
        _LIBMOD.check(self.lib.dsr_traffic_workspace_bytes(C.byref(self.params), C.byref(ws)),
                      "dsr_traffic_workspace_bytes")
        self.workspace = torch.empty(ws.value, dtype=torch.uint8, device="cuda")
        v = torch.as_tensor(np.ascontiguousarray(v0, dtype=np.int8).reshape(-1)).cuda()
        h = C.c_void_p()
        _LIBMOD.check(self.lib.dsr_traffic_create(self.heap.handle, C.byref(self.params), C.c_void_p(v.data_ptr()),
                                            C.c_void_p(self.workspace.data_ptr()), _stream_ptr(stream), C.byref(h)),
                "dsr_traffic_create")
        self.handle = h
        self._v0 = v

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.dsr_traffic_destroy(self.handle)
            self.handle = None

    def step(self, n=1, stream=None):
        L.check(self.lib.dsr_traffic_step(self.handle, n, _stream_ptr(stream)), "dsr_traffic_step")

    def count(self):
        return int(self.heap.stats()["live_objects"][0])

    def events(self):
        """Cumulative (cars entered, cars that left, cars that moved, velocity sum)."""
        c = self.heap.counters()
        return tuple(int(c["app%d" % k]) for k in range(4))

    def dump(self):
        """(cars int32[n, 3] (road, x, v) sorted, sources int32[R or 0, 3] sorted)."""
        cars, _ = self.heap.dump(0)
        src, _ = self.heap.dump(1)
        return _sorted_rows(cars.view(np.int32)), _sorted_rows(src.view(np.int32))

    def hash(self):
        return self.heap.hash(0), self.heap.hash(1)

    def occupancy(self):
        g = C.c_void_p()
        L.check(self.lib.dsr_traffic_occupancy(self.handle, C.byref(g)), "dsr_traffic_occupancy")
        n = self.R * self.L
        off = g.value - self.workspace.data_ptr()
        return self.workspace[off:off + n].cpu().numpy().reshape(self.R, self.L)


class Sugarscape:
    """Sugarscape (Epstein-Axtell rules M, G_alpha, R) on a W x H torus,
    driven through libdsr (rules in include/dsr_apps.h).

    cap: uint8[H, W] capacities (0..4); agents0: int32[n, 7] (x, y, sugar,
    metabolism, vision, age, max_age) at distinct cells.
    """

    def __init__(self, W, H, cap, agents0, seed, alpha=1, endow=(5, 25), metab=(1, 4), vision=(1, 6),
                 max_age=(60, 100), heap_bytes=None, tuning=None, stream=None):
        a0 = np.ascontiguousarray(agents0, dtype=np.int32).reshape(-1, 7)
        if len(a0):  # the kernels assume one agent per cell, on the torus
            if (a0[:, 0] < 0).any() or (a0[:, 0] >= W).any() or (a0[:, 1] < 0).any() or (a0[:, 1] >= H).any():
                raise ValueError("agent outside the W x H torus")
            if len(np.unique(a0[:, 1].astype(np.int64) * W + a0[:, 0])) != len(a0):
                raise ValueError("two agents on one cell")
        if np.asarray(cap).size != W * H:
            raise ValueError("cap must have W * H cells")
        self.lib = L.load()
        self.W, self.H = W, H
        self.params = L.SugarscapeParams(W, H, seed, alpha, endow[0], endow[1], metab[0], metab[1], vision[0],
                                         vision[1], max_age[0], max_age[1])
        if heap_bytes is None:
            heap_bytes = heap_bytes_for_blocks(SUGAR_TYPES, _blocks_for(len(a0) + 64, [64], tuning=tuning), tuning)
        self.heap = Heap(SUGAR_TYPES, heap_bytes, names=["Agent"], tuning=tuning, stream=stream)
        ws = C.c_size_t(0)
        L.check(self.lib.dsr_sugarscape_workspace_bytes(self.heap.handle, C.byref(self.params), C.byref(ws)),
                "dsr_sugarscape_workspace_bytes")
        self.workspace = torch.empty(ws.value, dtype=torch.uint8, device="cuda")
        c = torch.as_tensor(np.ascontiguousarray(cap, dtype=np.uint8).reshape(-1)).cuda()
        a = torch.as_tensor(a0.reshape(-1)).cuda() if len(a0) else torch.zeros(1, dtype=torch.int32, device="cuda")
        h = C.c_void_p()
        L.check(self.lib.dsr_sugarscape_create(self.heap.handle, C.byref(self.params), C.c_void_p(c.data_ptr()),
                                               C.c_void_p(a.data_ptr()), len(a0),
                                               C.c_void_p(self.workspace.data_ptr()), _stream_ptr(stream),
                                               C.byref(h)), "dsr_sugarscape_create")
        self.handle = h
        self._keep = (c, a)

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.dsr_sugarscape_destroy(self.handle)
            self.handle = None

    def step(self, n=1, stream=None):
        L.check(self.lib.dsr_sugarscape_step(self.handle, n, _stream_ptr(stream)), "dsr_sugarscape_step")

    def count(self):
        return int(self.heap.stats()["live_objects"][0])

    def events(self, stream=None):
        """Cumulative (moves, starved, aged, replacements placed elsewhere, sugar harvested)."""
        out = (C.c_uint64 * 5)()
        L.check(self.lib.dsr_sugarscape_events(self.handle, _stream_ptr(stream), out), "dsr_sugarscape_events")
        return tuple(int(v) for v in out)

    def dump(self):
        """(agents int32[n, 8] sorted, sugar int32[H, W])."""
        a, _ = self.heap.dump(0)
        sg = torch.empty(self.W * self.H, dtype=torch.int32, device="cuda")
        L.check(self.lib.dsr_sugarscape_sugar(self.handle, C.c_void_p(sg.data_ptr()), _stream_ptr()),
                "dsr_sugarscape_sugar")
        return _sorted_rows(a.view(np.int32)), sg.cpu().numpy().reshape(self.H, self.W)

    def hash(self):
        return self.heap.hash(0)
