"""Autotuner for the heap and do-all knobs.

The knobs (all in dsr_tuning, include/dsr.h):

  threads  threads per CTA of the do-all method kernels (64 .. 1024)
  cap_min  slots per block of the smallest type, 64 (as in Section 2) or 32
  fanout   bits used per bitmap container, 64 (Section 2.1), 32 or 16

None of them changes what a program computes (placement is free; results
are a function of the application rules), only how fast. The tuner measures
a caller-supplied workload under candidate settings and keeps the fastest.
Search: start from the defaults, then improve one knob at a time over its
values (coordinate descent), in the order threads, cap_min, fanout, for a
bounded number of passes. Results are cached in a JSON file keyed by device
name and workload key.
"""
import json
import os

DEFAULT = {"threads": 256, "cap_min": 64, "fanout": 64}
SPACE = {"threads": [128, 256, 512], "cap_min": [64, 32], "fanout": [64, 32, 16]}
ORDER = ("threads", "cap_min", "fanout")
CACHE = os.environ.get("DSR_AUTOTUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json"))


def _key(t):
    return tuple(t[k] for k in ORDER)


def search(measure, space=None, start=None, passes=2):
    """Coordinate descent over `space`.

    measure(tuning) -> throughput (higher is better), or None when the
    setting cannot run (it is then skipped). Returns (best tuning, best
    throughput, {setting tuple: throughput} of every setting measured).
    Each setting is measured once.
    """
    space = space or SPACE
    best = dict(start or DEFAULT)
    seen = {}

    def score(t):
        k = _key(t)
        if k not in seen:
            seen[k] = measure(dict(t))
        return seen[k]

    best_v = score(best)
    if best_v is None:
        raise RuntimeError("the starting setting %s cannot run" % best)
    for _ in range(passes):
        improved = False
        for knob in ORDER:
            for v in space[knob]:
                if v == best[knob]:
                    continue
                cand = dict(best, **{knob: v})
                s = score(cand)
                if s is not None and s > best_v:
                    best, best_v, improved = cand, s, True
        if not improved:
            break
    return best, best_v, seen


def load_cache(path=CACHE):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(key, tuning, value, table, path=CACHE):
    """Record a result under `key` (device name / workload)."""
    c = load_cache(path)
    c[key] = {"tuning": tuning, "value": value,
              "table": {",".join(str(x) for x in k): v for k, v in table.items()}}
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned(key, measure, space=None, path=CACHE, refresh=False):
    """The cached best tuning for `key`, or a fresh search (then cached)."""
    if not refresh:
        hit = load_cache(path).get(key)
        if hit:
            return hit["tuning"], hit["value"], None
    best, v, table = search(measure, space)
    store(key, best, v, table, path)
    return best, v, table


def wator_batch_measure(sides, seeds, steps=5, warmup=2):
    """A measure() for the batched wa-tor form: builds the instances under
    the candidate tuning, steps them `warmup` times, then times `steps`
    graph-captured steps with CUDA events; object-updates/s."""
    import torch

    from . import workloads as WL
    from .apps import WatorBatch

    def measure(t):
        tun = {"threads": t["threads"], "cap_min": t["cap_min"], "fanout": t["fanout"]}
        need = sum(WatorBatch.blocks_for(s, s) * 1100 + s * s * 24 for s in sides) + (64 << 20)
        b = WatorBatch(need, max_instances=len(sides), tuning=tun)
        slots = []
        for s, sd in zip(sides, seeds):
            x = b.add(int(s), int(s), WL.wator_initial(int(s), int(s), int(sd)), int(sd))
            if x is None:
                return None
            slots.append(x)
        b.step(warmup)
        torch.cuda.synchronize()
        v0 = sum(b.heap(x).counters()["visits"] for x in slots)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.step(steps)
        e1.record()
        e1.synchronize()
        v1 = sum(b.heap(x).counters()["visits"] for x in slots)
        err = any(b.heap(x).stats()["error_flags"] for x in slots)
        del b
        torch.cuda.empty_cache()
        if err:
            return None
        return (v1 - v0) / (e0.elapsed_time(e1) * 1e-3)

    return measure
