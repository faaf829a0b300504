"""Python binding of the heap C ABI (include/dsr.h): argument marshalling only.

PyTorch provides the device memory (the arena and output buffers) and the
stream; every step of the allocator and the do-all runs in libdsr.so.
"""
import ctypes as C

import numpy as np
import torch

from . import _lib as L


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _descs(types, names=None):
    arrs = [(C.c_int * len(t))(*t) for t in types]
    descs = (L.TypeDesc * len(types))()
    for i, t in enumerate(types):
        descs[i].name = (names[i] if names else "T%d" % i).encode()
        descs[i].n_fields = len(t)
        descs[i].field_bytes = C.cast(arrs[i], C.POINTER(C.c_int))
    return descs, arrs


def _tuning(t):
    if t is None:
        return None
    return L.Tuning(int(t.get("cap_min", 0)), int(t.get("threads", 0)), int(t.get("ctas_per_sm", 0)),
                    int(t.get("fanout", 0)))


def heap_bytes_for_blocks(types, n_blocks, tuning=None):
    """Arena bytes that give at least n_blocks blocks for these types (list of field-byte lists)."""
    lib = L.load()
    descs, _keep = _descs(types)
    out = C.c_size_t(0)
    tun = _tuning(tuning)
    L.check(lib.dsr_heap_bytes_for_blocks(descs, len(types), n_blocks, C.byref(tun) if tun else None,
                                          C.byref(out)), "dsr_heap_bytes_for_blocks")
    return int(out.value)


def type_tree(types, bases):
    """Bit masks of the types a do-all over each type visits, given each
    type's direct base (-1 for none); raises DsrError for an invalid
    hierarchy (a base after its subtype, or leading fields that differ)."""
    lib = L.load()
    descs, _keep = _descs(types)
    b = (C.c_int * len(types))(*bases)
    out = (C.c_uint32 * len(types))()
    L.check(lib.dsr_type_tree(descs, len(types), b, out), "dsr_type_tree")
    return [int(x) for x in out]


class Heap:
    """A dsr heap in a torch-allocated device arena.

    types: list of per-type field byte sizes, e.g. [[4, 4, 4], [4, 4, 4, 4]].
    bases: optional direct base type of each type (-1 for none); a do-all
    over a type then also visits its subtypes' objects.
    """

    def __init__(self, types, heap_bytes, names=None, tuning=None, stream=None, device="cuda", bases=None):
        self.lib = L.load()
        self.types = [list(t) for t in types]
        self.names = names
        self.tuning = tuning
        self.arena = torch.empty(int(heap_bytes), dtype=torch.uint8, device=device)
        descs, keep = _descs(self.types, names)
        self._keep = (descs, keep)
        tun = _tuning(tuning)
        h = C.c_void_p()
        L.check(self.lib.dsr_heap_create(descs, len(types), C.c_void_p(self.arena.data_ptr()), int(heap_bytes),
                                         C.byref(tun) if tun else None, _stream_ptr(stream), C.byref(h)),
                "dsr_heap_create")
        self.handle = h
        self._scratch = torch.zeros(2, dtype=torch.int64, device=device)
        if bases is not None:
            self.set_bases(bases)

    def set_bases(self, bases):
        """Declare each type's direct base (-1 for none); see type_tree."""
        b = (C.c_int * len(self.types))(*bases)
        L.check(self.lib.dsr_heap_set_bases(self.handle, b), "dsr_heap_set_bases")

    @classmethod
    def view(cls, handle, types, arena, names=None):
        """A non-owning wrapper of a heap that lives inside another object (a group)."""
        h = cls.__new__(cls)
        h.lib = L.load()
        h.types = [list(t) for t in types]
        h.names = names
        h.arena = arena  # a tensor whose memory begins with the heap (for snapshot offsets)
        h.handle = C.c_void_p(handle.value if isinstance(handle, C.c_void_p) else handle)
        h._owner = False
        h._scratch = torch.zeros(2, dtype=torch.int64, device="cuda")
        return h

    def close(self):
        if getattr(self, "handle", None) and getattr(self, "_owner", True):
            self.lib.dsr_heap_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- inspection ---------------------------------------------------------
    def layout(self):
        lay = L.Layout()
        L.check(self.lib.dsr_heap_layout(self.handle, C.byref(lay)), "dsr_heap_layout")
        return lay

    def capacity(self, t):
        return int(self.layout().capacity[t])

    def stats(self, stream=None):
        st = L.Stats()
        L.check(self.lib.dsr_heap_stats(self.handle, _stream_ptr(stream), C.byref(st)), "dsr_heap_stats")
        n = st.n_types
        return {
            "n_blocks": int(st.n_blocks),
            "free_blocks": int(st.free_blocks),
            "error_flags": int(st.error_flags),
            "capacity": [int(st.capacity[t]) for t in range(n)],
            "live_objects": [int(st.live_objects[t]) for t in range(n)],
            "allocated_blocks": [int(st.allocated_blocks[t]) for t in range(n)],
            "active_blocks": [int(st.active_blocks[t]) for t in range(n)],
        }

    def counters(self, stream=None):
        """Cumulative event counts: visits, allocs, frees, blocks taken from
        free, and the application counters app0..app3 (wa-tor: app0 counts
        successful moves)."""
        out = (C.c_uint64 * L.CTR_COUNT)()
        L.check(self.lib.dsr_heap_counters(self.handle, _stream_ptr(stream), out), "dsr_heap_counters")
        d = {"visits": int(out[0]), "allocs": int(out[1]), "frees": int(out[2]), "new_blocks": int(out[3])}
        for k in range(4, L.CTR_COUNT):
            d["app%d" % (k - 4)] = int(out[k])
        return d

    def snapshot(self):
        """Metadata of a quiescent heap as numpy arrays (for the invariant checker)."""
        torch.cuda.synchronize()
        lay = self.layout()
        meta = self.arena[: lay.off_data].cpu().numpy()
        M, W, T = int(lay.n_blocks), int(lay.bitmap_words), int(lay.n_types)

        def u64(off, n):
            return meta[off: off + 8 * n].view(np.uint64).copy()

        return {
            "M": M,
            "capacity": np.array([lay.capacity[t] for t in range(T)], dtype=np.uint32),
            "obj_free": u64(lay.off_obj, M),
            "block_type": meta[lay.off_type: lay.off_type + M].copy(),
            "free_bm": u64(lay.off_free_bm, W),
            "alloc_bm": u64(lay.off_alloc_bm, T * W).reshape(T, W),
            "active_bm": u64(lay.off_active_bm, T * W).reshape(T, W),
            "words_per_level": np.array([lay.words_per_level[l] for l in range(lay.n_levels)], dtype=np.uint64),
            "width": int(lay.fanout),
        }

    # -- do-all -------------------------------------------------------------
    def parallel_do(self, type_id, method, args=None, stream=None):
        if args is None:
            ptr, n = None, 0
        else:
            ptr, n = C.cast(C.byref(args), C.c_void_p), C.sizeof(args)
        L.check(self.lib.dsr_parallel_do(self.handle, type_id, method, ptr, n, _stream_ptr(stream)),
                "dsr_parallel_do")

    def count(self, type_id, stream=None):
        """Number of objects a do-all over type_id visits (method COUNT)."""
        self._scratch.zero_()
        self.parallel_do(type_id, L.METHOD_COUNT, L.CountArgs(C.c_void_p(self._scratch.data_ptr())), stream)
        return int(self._scratch[0].item())

    def dump(self, type_id, cap=None, stream=None):
        """(fields uint32[n, words], handles uint64[n]) of the live objects of a type, in arbitrary order."""
        row = self.lib.dsr_row_words(self.handle, type_id)
        if row < 0:
            raise L.DsrError("bad type id")
        if cap is None:
            lay = self.layout()
            cap = int(lay.n_blocks) * int(lay.capacity[type_id])
        out = torch.empty(max(cap, 1) * row, dtype=torch.int32, device=self.arena.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=self.arena.device)
        L.check(self.lib.dsr_heap_dump(self.handle, type_id, C.c_void_p(out.data_ptr()), cap,
                                       C.c_void_p(cnt.data_ptr()), _stream_ptr(stream)), "dsr_heap_dump")
        n = int(cnt.item())
        if n > cap:
            raise L.DsrError("dump capacity %d < %d objects" % (cap, n))
        a = out[: n * row].cpu().numpy().view(np.uint32).reshape(n, row)
        handles = a[:, -2].astype(np.uint64) | (a[:, -1].astype(np.uint64) << np.uint64(32))
        return a[:, :-2].copy(), handles

    def hash(self, type_id, stream=None):
        self._scratch.zero_()
        L.check(self.lib.dsr_heap_hash(self.handle, type_id, C.c_void_p(self._scratch.data_ptr()),
                                       _stream_ptr(stream)), "dsr_heap_hash")
        return int(self._scratch[0].item()) & 0xFFFFFFFFFFFFFFFF

    def reset(self, stream=None):
        L.check(self.lib.dsr_heap_reset(self.handle, _stream_ptr(stream)), "dsr_heap_reset")

    def inject_oom(self, n, stream=None):
        L.check(self.lib.dsr_heap_inject_oom(self.handle, n, _stream_ptr(stream)), "dsr_heap_inject_oom")

    # -- microbenchmark kernels ----------------------------------------------
    def bench_alloc(self, refs, n_types_used, seed, stream=None):
        L.check(self.lib.dsr_bench_alloc(self.handle, refs.numel(), n_types_used, seed,
                                         C.c_void_p(refs.data_ptr()), _stream_ptr(stream)), "dsr_bench_alloc")

    def bench_free(self, refs, stream=None):
        L.check(self.lib.dsr_bench_free(self.handle, refs.numel(), C.c_void_p(refs.data_ptr()),
                                        _stream_ptr(stream)), "dsr_bench_free")


class BitmapHeap:
    """A BitmapAlloc comparator heap (dsr_bm_heap_*): per type, an array of
    capacity[T] objects stored as structs and a flat bitmap of its slots."""

    def __init__(self, types, capacity, stream=None, device="cuda"):
        self.lib = L.load()
        self.types = [list(t) for t in types]
        descs, keep = _descs(self.types)
        self._keep = (descs, keep)
        cap = (C.c_uint64 * len(types))(*[int(c) for c in capacity])
        self._cap = cap
        n = C.c_size_t(0)
        L.check(self.lib.dsr_bm_heap_bytes(descs, len(types), cap, C.byref(n)), "dsr_bm_heap_bytes")
        self.arena = torch.empty(n.value, dtype=torch.uint8, device=device)
        h = C.c_void_p()
        L.check(self.lib.dsr_bm_heap_create(descs, len(types), cap, C.c_void_p(self.arena.data_ptr()), n.value,
                                            _stream_ptr(stream), C.byref(h)), "dsr_bm_heap_create")
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.dsr_bm_heap_destroy(self.handle)
            self.handle = None

    def stats(self, stream=None):
        live = (C.c_uint64 * len(self.types))()
        err = C.c_uint32(0)
        L.check(self.lib.dsr_bm_heap_stats(self.handle, _stream_ptr(stream), live, C.byref(err)), "dsr_bm_heap_stats")
        return {"live_objects": [int(x) for x in live], "error_flags": int(err.value)}

    def hash(self, type_id, stream=None):
        out = torch.zeros(1, dtype=torch.int64, device=self.arena.device)
        L.check(self.lib.dsr_bm_heap_hash(self.handle, type_id, C.c_void_p(out.data_ptr()), _stream_ptr(stream)),
                "dsr_bm_heap_hash")
        return int(out.cpu().numpy().view(np.uint64)[0])

    def counters(self, stream=None):
        out = (C.c_uint64 * L.CTR_COUNT)()
        L.check(self.lib.dsr_bm_heap_counters(self.handle, _stream_ptr(stream), out), "dsr_bm_heap_counters")
        d = {"visits": int(out[0]), "allocs": int(out[1]), "frees": int(out[2]), "new_blocks": int(out[3])}
        for k in range(4, L.CTR_COUNT):
            d["app%d" % (k - 4)] = int(out[k])
        return d
