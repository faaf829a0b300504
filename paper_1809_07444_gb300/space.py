"""Space efficiency (Section 4, "Space Efficiency"; Fig. 8).

Every allocator gets the same heap size, and the experiment finds the
largest problem the application runs without running out of memory. Here the
application is wa-tor (square torus, the bench's densities and rules), the
problem size is the side of the torus, and the search is a bisection over
the side. A run fits when `steps` steps end with no DSR_ERR_OOM (or
DSR_ERR_RETRY) and the heap could be created at all.

Reported beside the largest side: the peak bytes of live object data during
that run (12 B per fish, 16 B per shark) and its fraction of the heap, the
space efficiency.
"""
import ctypes as C

import torch

from . import _lib as L
from . import workloads as WL
from .apps import Wator

OBJECT_BYTES = (12, 16)  # Fish {x, y, timer}, Shark {x, y, timer, energy}


def wator_fits(side, heap_bytes, steps, seed=1, tuning=None):
    """(fits, peak live object bytes) of one run."""
    try:
        w = Wator(side, side, WL.wator_initial(side, side, seed), seed, heap_bytes=heap_bytes, tuning=tuning)
    except L.DsrError:
        return False, 0  # the heap holds no block, or too few for the first agents
    peak = 0
    ok = True
    for _ in range(steps):
        w.step(1)
        st = w.heap.stats()
        if st["error_flags"] & (L.ERR_OOM | L.ERR_RETRY):
            ok = False
            break
        live = st["live_objects"]
        peak = max(peak, live[0] * OBJECT_BYTES[0] + live[1] * OBJECT_BYTES[1])
    del w
    torch.cuda.empty_cache()
    return ok, peak


def _bisect(fits, lo=8, hi=None):
    """Largest side (to within 1) with fits(side)[0], and that run's peak."""
    if hi is None:
        hi = 16
        while fits(hi)[0]:
            lo, hi = hi, hi * 2
    ok, peak = fits(lo)
    if not ok:
        return 0, 0
    best, best_peak = lo, peak
    while hi - lo > 1:
        mid = (lo + hi) // 2
        ok, peak = fits(mid)
        if ok:
            lo, best, best_peak = mid, mid, peak
        else:
            hi = mid
    return best, best_peak


def max_wator_side(heap_bytes, steps=100, seed=1, tuning=None, lo=8, hi=None):
    """Largest side (to within 1) that fits, with that run's peak live bytes."""
    return _bisect(lambda s: wator_fits(s, heap_bytes, steps, seed, tuning), lo, hi)


def bitmap_capacities(heap_bytes, fish_share):
    """BitmapAlloc slot counts that split heap_bytes between the Fish and
    Shark arrays (fish_share of the object bytes to fish), the largest that
    fit heap_bytes with the comparator's bitmaps and header."""
    from .apps import WATOR_TYPES
    from .heap import _descs
    lib = L.load()
    descs, _keep = _descs(WATOR_TYPES)
    scale = 1.0
    while scale > 0.5:
        cf = max(64, int(scale * fish_share * heap_bytes / OBJECT_BYTES[0]) // 64 * 64)
        cs = max(64, int(scale * (1 - fish_share) * heap_bytes / OBJECT_BYTES[1]) // 64 * 64)
        n = C.c_size_t(0)
        cap = (C.c_uint64 * 2)(cf, cs)
        L.check(lib.dsr_bm_heap_bytes(descs, 2, cap, C.byref(n)), "dsr_bm_heap_bytes")
        if n.value <= heap_bytes:
            return [cf, cs]
        scale -= 0.002
    return [64, 64]


def wator_bitmap_fits(side, heap_bytes, steps, fish_share, seed=1):
    """(fits, peak live object bytes) on the BitmapAlloc comparator."""
    from .apps import WatorBitmap
    w = WatorBitmap(side, side, WL.wator_initial(side, side, seed), seed,
                    capacity=bitmap_capacities(heap_bytes, fish_share))
    peak, ok = 0, True
    for _ in range(steps):
        w.step(1)
        st = w.heap.stats()
        if st["error_flags"] & (L.ERR_OOM | L.ERR_RETRY):
            ok = False
            break
        live = st["live_objects"]
        peak = max(peak, live[0] * OBJECT_BYTES[0] + live[1] * OBJECT_BYTES[1])
    del w
    torch.cuda.empty_cache()
    return ok, peak


def experiment(heap_bytes=32 << 20, steps=100, tunings=None, bitmap=True, seed=1):
    """The largest wa-tor side per allocator setting, with the space efficiency.

    dsr rows: one per tuning. BitmapAlloc rows: the heap split between the
    Fish and Shark arrays (a) by the initial population's bytes, which is what
    a user can know in advance, and (b) by the peak bytes of each type in a
    dsr run of the same rules on a 256 x 256 torus (hindsight), about the
    best a fixed split can do.
    """
    tunings = tunings or [None, {"cap_min": 32}, {"fanout": 16}]
    rows = []
    for t in tunings:
        side, peak = max_wator_side(heap_bytes, steps, seed=seed, tuning=t)
        rows.append({"allocator": "dsr", "tuning": t or "default", "max_side": side, "peak_live_bytes": peak,
                     "efficiency": peak / heap_bytes})
    if bitmap:
        k0 = WL.wator_initial(256, 256, seed)
        b0 = [int((k0 == 1).sum()) * OBJECT_BYTES[0], int((k0 == 2).sum()) * OBJECT_BYTES[1]]
        w = Wator(256, 256, k0, seed)
        pk = [0, 0]
        for _ in range(steps):
            w.step(1)
            live = w.heap.stats()["live_objects"]
            pk = [max(pk[0], live[0] * OBJECT_BYTES[0]), max(pk[1], live[1] * OBJECT_BYTES[1])]
        del w
        for name, share in (("initial split", b0[0] / sum(b0)), ("hindsight split", pk[0] / sum(pk))):
            side, peak = _bisect(lambda s: wator_bitmap_fits(s, heap_bytes, steps, share, seed))
            rows.append({"allocator": "BitmapAlloc", "tuning": "%s (fish %.3f)" % (name, share), "max_side": side,
                         "peak_live_bytes": peak, "efficiency": peak / heap_bytes})
    return {"app": "wa-tor", "heap_bytes": heap_bytes, "steps": steps, "rows": rows}
