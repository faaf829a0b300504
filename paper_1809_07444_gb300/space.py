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


def max_wator_side(heap_bytes, steps=100, seed=1, tuning=None, lo=8, hi=None):
    """Largest side (to within 1) that fits, with that run's peak live bytes."""
    if hi is None:
        hi = 16
        while wator_fits(hi, heap_bytes, steps, seed, tuning)[0]:
            lo, hi = hi, hi * 2
    best, best_peak = None, 0
    ok, peak = wator_fits(lo, heap_bytes, steps, seed, tuning)
    if not ok:
        return 0, 0
    best, best_peak = lo, peak
    while hi - lo > 1:
        mid = (lo + hi) // 2
        ok, peak = wator_fits(mid, heap_bytes, steps, seed, tuning)
        if ok:
            lo, best, best_peak = mid, mid, peak
        else:
            hi = mid
    return best, best_peak


def experiment(heap_bytes=32 << 20, steps=100, tunings=None):
    """The largest wa-tor side per tuning, with the space efficiency."""
    tunings = tunings or [None, {"cap_min": 32}, {"fanout": 16}]
    rows = []
    for t in tunings:
        side, peak = max_wator_side(heap_bytes, steps, tuning=t)
        rows.append({"tuning": t or "default", "max_side": side, "peak_live_bytes": peak,
                     "efficiency": peak / heap_bytes})
    return {"app": "wa-tor", "heap_bytes": heap_bytes, "steps": steps, "rows": rows}
