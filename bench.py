#!/usr/bin/env python
"""Benchmark of the dsr hot path: one JSON line on rank 0.

Workload: wa-tor on a 2048 x 2048 torus (30% fish, 3% sharks, seed 1), the
plain one-simulation form. A step is one wa-tor step: five parallel do-alls
(scan + compaction + method kernel each) with device new/delete for births
and deaths, i.e. every row of the hot path.

  value      do-all object-updates/s (objects visited by method kernels per
             second of device time), inputs resident in HBM;
  e2e        the same metric through the C ABI with the initial grid in
             pinned host memory: host->device copy, heap reset, agent
             creation, the K steps and the device->host read of the final
             state hash all inside the timed region;
  roofline   the fish-choice method kernel (the largest share of a step),
             algorithmic bytes / its CUDA-event time, against the measured
             HBM copy peak;
  cpu_baseline  the oracle (single-threaded C++) on the same workload.

L2 (129 MB) is flushed by writing a 512 MB buffer before every timed step,
outside the step's events. Multi-GPU: one independent replica per rank (no
data exchange), weak scaling.

--impl reference times the oracle instead, on the host cores of rank 0.
"""
import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "alloc+free/s & do-all object-updates/s on 1 GB300, batched vs plain; %HBM peak"
UNIT = "object-updates/s"
W_SIDE = 2048
SEED = 1
WORKLOAD = {"workload": "wator-2048x2048", "grid": [W_SIDE, W_SIDE], "fish": 0.30, "sharks": 0.03,
            "fish_breed": 3, "shark_breed": 10, "shark_energy0": 5, "shark_gain": 3, "seed": SEED,
            "form": "plain (one simulation per launch sequence)", "l2": "flushed before every timed step"}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="dsr", choices=["dsr", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-extra", action="store_true", help="headline only (no batched/served/microbenchmarks)")
    p.add_argument("--served-seconds", type=float, default=20.0)
    return p.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# oracle timing (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def oracle_wator_rate(seconds, steps=None, warmup=0):
    """Object-updates/s of the oracle's wa-tor on the bench workload.

    Runs `warmup` untimed steps, then steps until `steps` are done (if given)
    or `seconds` have passed. Updates per step are the objects each of its
    five do-alls visits: 2 x fish + sharks + 2 x (sharks that did not starve).
    """
    import oracle as O
    from paper_1809_07444_gb300 import workloads as WL

    k0 = WL.wator_initial(W_SIDE, W_SIDE, SEED)
    w = O.Wator(W_SIDE, W_SIDE, k0, seed=SEED)
    if warmup:
        w.step(warmup)
    updates, n, t0 = 0, 0, time.perf_counter()
    while True:
        nf, ns = w.counts()
        ev = w.step(1)[0]
        updates += 2 * nf + ns + 2 * (ns - int(ev[3]))
        n += 1
        el = time.perf_counter() - t0
        if (steps is not None and n >= steps) or (steps is None and el >= seconds):
            break
    return updates / el, n, el


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def fish_choice_bytes(n_fish, n_blocks, cells):
    """Algorithmic bytes of one fish-choice (F1) method kernel launch.

    Per fish: x, y, timer read (12 B) and timer written (4 B), the intent
    word written (4 B), one claim word read-modify-written (16 B, at most one
    per fish); per listed block its R entry (12 B); and the grid read once
    (8 B per cell), since every cell neighbours some fish at this density.
    """
    return n_fish * (12 + 4 + 4 + 16) + n_blocks * 12 + cells * 8


def run_gpu(args, rank, world):
    import numpy as np
    import torch

    from paper_1809_07444_gb300 import _lib as L
    from paper_1809_07444_gb300 import workloads as WL
    from paper_1809_07444_gb300.apps import Wator
    from paper_1809_07444_gb300.heap import _stream_ptr

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    lib = L.load()
    seed = SEED + rank
    k0 = WL.wator_initial(W_SIDE, W_SIDE, seed)
    sim = Wator(W_SIDE, W_SIDE, k0, seed)
    stream = torch.cuda.current_stream()
    sp = _stream_ptr(stream)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up
    for _ in range(args.warmup):
        L.check(lib.dsr_wator_step(sim.handle, 1, sp), "dsr_wator_step")
    torch.cuda.synchronize()
    c0 = sim.heap.counters()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    with Clocks(dev) as clk:
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            evs[k][0].record(stream)
            L.check(lib.dsr_wator_step(sim.handle, 1, sp), "dsr_wator_step")
            evs[k][1].record(stream)
        barrier()
    c1 = sim.heap.counters()
    dev_s = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    visits = c1["visits"] - c0["visits"]
    allocfree = (c1["allocs"] - c0["allocs"]) + (c1["frees"] - c0["frees"])
    st = sim.heap.stats()
    if st["error_flags"]:
        raise RuntimeError("device error flags %d" % st["error_flags"])

    # Per-phase method-kernel timing, after the timed region (the state keeps
    # advancing): L2 flushed before each step, scan outside the events, the
    # objects visited and blocks listed read back between scan and run.
    methods = [(0, L.METHOD_WATOR_F1), (0, L.METHOD_WATOR_F2), (1, L.METHOD_WATOR_S0), (1, L.METHOD_WATOR_S1),
               (1, L.METHOD_WATOR_S2)]
    wh = C.c_void_p(sim.handle.value)
    phases = {i: [] for i in range(len(methods))}
    for rep in range(5):
        flush.fill_(rep)
        for i, (t, m) in enumerate(methods):
            v0 = sim.heap.counters()["visits"]
            L.check(lib.dsr_doall_scan(sim.heap.handle, t, sp), "dsr_doall_scan")
            torch.cuda.synchronize()
            objs = sim.heap.counters()["visits"] - v0
            nblocks = int(sim.heap.arena[8:12].cpu().view(torch.int32).item())  # R length in the heap header
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            L.check(lib.dsr_doall_run(sim.heap.handle, t, m, C.byref(wh), C.sizeof(wh), sp), "dsr_doall_run")
            b.record(stream)
            b.synchronize()
            phases[i].append((a.elapsed_time(b), objs, nblocks))
    med = {i: statistics.median(x[0] for x in v) for i, v in phases.items()}
    f1 = phases[0]
    f1_gbs = statistics.median(fish_choice_bytes(o, nb, W_SIDE * W_SIDE) / (ms * 1e-3) / 1e9 for ms, o, nb in f1)
    f1_bytes = statistics.median(fish_choice_bytes(o, nb, W_SIDE * W_SIDE) for ms, o, nb in f1)

    # e2e through the C ABI with host buffers
    k0_host = torch.from_numpy(np.ascontiguousarray(k0.reshape(-1))).pin_memory()
    k0_dev = torch.empty_like(k0_host, device="cuda")
    hash_dev = torch.zeros(2, dtype=torch.int64, device="cuda")
    hash_host = torch.zeros(2, dtype=torch.int64).pin_memory()
    ws = sim.workspace
    params = sim.params
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_host0 = time.perf_counter()
    e0.record(stream)
    k0_dev.copy_(k0_host, non_blocking=True)
    L.check(lib.dsr_heap_reset(sim.heap.handle, sp), "dsr_heap_reset")
    h2 = C.c_void_p()
    L.check(lib.dsr_wator_create(sim.heap.handle, C.byref(params), C.c_void_p(k0_dev.data_ptr()),
                                 C.c_void_p(ws.data_ptr()), sp, C.byref(h2)), "dsr_wator_create")
    L.check(lib.dsr_wator_step(h2, args.steps, sp), "dsr_wator_step")
    hash_dev.zero_()
    L.check(lib.dsr_heap_hash(sim.heap.handle, 0, C.c_void_p(hash_dev.data_ptr()), sp), "dsr_heap_hash")
    hash_host.copy_(hash_dev, non_blocking=True)
    e1.record(stream)
    e1.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    lib.dsr_wator_destroy(h2)
    c2 = sim.heap.counters()  # counters restarted at the reset
    hashed = sim.heap.stats()["live_objects"][0]  # objects the final hash do-all visited
    return {
        "dev_s": dev_s, "visits": visits, "allocfree": allocfree, "clocks": clk.summary(),
        "phase_ms": med, "f1_gbs": f1_gbs, "f1_bytes": f1_bytes, "f1_ms": med[0], "e2e_s": e2e_s, "e2e_visits": c2["visits"] - hashed,
        "h2d": k0_host.numel(), "d2h": 16, "stats": st,
    }


# ---------------------------------------------------------------------------
# secondary measurements (rank 0, after the headline)
# ---------------------------------------------------------------------------
def _ev():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def bench_alloc_free(n=1 << 24, n_types=2, reps=3):
    """Allocation microbenchmark: n threads each create one object (types by a
    hash of the thread index), then every object is deleted; fresh heap, L2
    flushed before each timed kernel."""
    import torch
    from paper_1809_07444_gb300.heap import Heap, heap_bytes_for_blocks

    types = [[4, 4], [4, 4, 4, 4]]
    h = Heap(types, heap_bytes_for_blocks(types, int(n / 32 * 1.3) + 4096))
    refs = torch.empty(n, dtype=torch.int64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ta, tf = [], []
    for r in range(reps + 1):
        h.reset()
        flush.fill_(r)
        a0, a1 = _ev()
        a0.record()
        h.bench_alloc(refs, n_types, 77 + r)
        a1.record()
        flush.fill_(r + 1)
        f0, f1 = _ev()
        f0.record()
        h.bench_free(refs)
        f1.record()
        torch.cuda.synchronize()
        if r:  # first round warms up
            ta.append(a0.elapsed_time(a1) / 1e3)
            tf.append(f0.elapsed_time(f1) / 1e3)
    st = h.stats()
    ok = st["error_flags"] == 0 and st["free_blocks"] == st["n_blocks"]
    return {"objects": n, "types": n_types, "allocs_per_s": n / statistics.median(ta),
            "frees_per_s": n / statistics.median(tf), "alloc_free_per_s": 2 * n / (statistics.median(ta) + statistics.median(tf)),
            "heap_consistent_after": ok, "l2": "flushed before each kernel"}


def bench_streaming_doall(n=1 << 28, fields=4, reps=5):
    """Streaming do-all: one type with `fields` int32 fields, n objects (>> L2);
    method field f += field f+1 (reads every field, writes every field)."""
    import torch
    from paper_1809_07444_gb300 import _lib as L
    from paper_1809_07444_gb300.heap import Heap, heap_bytes_for_blocks, _stream_ptr

    types = [[4] * fields]
    blocks = n // 64
    h = Heap(types, heap_bytes_for_blocks(types, blocks + 1024))
    refs = torch.empty(n, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 1, 5)
    del refs
    torch.cuda.synchronize()
    lib, sp = h.lib, _stream_ptr()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ms, ms_full = [], []
    for r in range(reps + 1):
        flush.fill_(r)
        L.check(lib.dsr_doall_scan(h.handle, 0, sp), "dsr_doall_scan")
        a0, a1 = _ev()
        a0.record()
        L.check(lib.dsr_doall_run(h.handle, 0, L.METHOD_STREAM_ADD, None, 0, sp), "dsr_doall_run")
        a1.record()
        flush.fill_(r + 1)
        b0, b1 = _ev()
        b0.record()
        h.parallel_do(0, L.METHOD_STREAM_ADD, None)
        b1.record()
        torch.cuda.synchronize()
        if r:
            ms.append(a0.elapsed_time(a1))
            ms_full.append(b0.elapsed_time(b1))
    st = h.stats()
    live = st["live_objects"][0]
    alloc_blocks = st["allocated_blocks"][0]
    # algorithmic bytes: every field read and written once, plus the R entry
    # (12 B) of each listed block
    bytes_method = live * fields * 4 * 2 + alloc_blocks * 12
    t = statistics.median(ms) * 1e-3
    peak, kind = _peaks()
    return {"objects": live, "fields": fields, "method_ms": t * 1e3, "doall_ms": statistics.median(ms_full),
            "object_updates_per_s": live / t, "achieved_gbs": bytes_method / t / 1e9, "peak_gbs": peak,
            "frac": bytes_method / t / 1e9 / peak, "peak_source": kind,
            "algorithmic_bytes": bytes_method, "fill": live / (alloc_blocks * 64)}


def bench_batched(n_inst=256, steps=20, one_by_one_steps=3):
    """The batched workload (256 wa-tor instances, sides log-uniform in
    [64, 1024]) advanced by graph-captured group steps, against the same
    instances stepped one by one in the plain form."""
    import torch
    from paper_1809_07444_gb300 import workloads as WL
    from paper_1809_07444_gb300.apps import Wator, WatorBatch

    sides = [int(s) for s in WL.batched_sides(n_inst, 1)]
    need = sum(WatorBatch.blocks_for(s, s) * 1000 + s * s * 24 for s in sides)
    b = WatorBatch(need + (256 << 20), max_instances=n_inst)
    slots = [b.add(s, s, WL.wator_initial(s, s, 1000 + i), 1000 + i) for i, s in enumerate(sides)]
    b.step(3)
    torch.cuda.synchronize()
    v0 = sum(b.heap(x).counters()["visits"] for x in slots)
    e0, e1 = _ev()
    e0.record()
    b.step(steps)
    e1.record()
    e1.synchronize()
    v1 = sum(b.heap(x).counters()["visits"] for x in slots)
    t_b = e0.elapsed_time(e1) / 1e3
    del b
    torch.cuda.empty_cache()
    plain = [Wator(s, s, WL.wator_initial(s, s, 1000 + i), 1000 + i) for i, s in enumerate(sides)]
    for w in plain:
        w.step(3)
    torch.cuda.synchronize()
    p0 = sum(w.heap.counters()["visits"] for w in plain)
    e0, e1 = _ev()
    e0.record()
    for _ in range(one_by_one_steps):
        for w in plain:
            w.step(1)
    e1.record()
    e1.synchronize()
    p1 = sum(w.heap.counters()["visits"] for w in plain)
    t_p = e0.elapsed_time(e1) / 1e3
    vb, vp = (v1 - v0) / t_b, (p1 - p0) / t_p
    return {"workload": "wator-batched-%d (sides log-uniform [64, 1024], seeds 1000+i)" % n_inst,
            "cells": int(sum(s * s for s in sides)), "steps": steps, "ms_per_step": t_b * 1e3 / steps,
            "object_updates_per_s": vb, "one_by_one": {"object_updates_per_s": vp, "steps": one_by_one_steps,
                                                       "ms_per_step": t_p * 1e3 / one_by_one_steps,
                                                       "launches_per_step": 10 * n_inst},
            "speedup_vs_one_by_one": vb / vp if vp else None, "launches_per_step": 10, "graph": True}


def bench_served(seconds=20.0, n_jobs=10000, arena_gb=64, lo=128, hi=4096, steps_lo=50, steps_hi=1000,
                 label="the 10,000-job stream"):
    """The served workload (Poisson 200 jobs/s, game-of-life and wa-tor, sides
    log-uniform in [lo, hi], steps uniform in [steps_lo, steps_hi], arenas of
    arena_gb GB), in real time for at most `seconds` of wall time."""
    import torch
    from paper_1809_07444_gb300 import workloads as WL
    from paper_1809_07444_gb300.serve import Server, summarize

    s = WL.served_jobs(n_jobs, 2024, lo=lo, hi=hi, steps_lo=steps_lo, steps_hi=steps_hi)
    jobs = [{"id": i, "arrival": float(s["arrival"][i]), "app": int(s["app"][i]), "side": int(s["side"][i]),
             "steps": int(s["steps"][i]), "seed": int(s["seed"][i])} for i in range(n_jobs)]
    srv = Server(arena_bytes=arena_gb << 30, max_jobs=4096)
    rep = srv.run(jobs, time_limit=seconds, realtime=True, keep_hashes=False)
    out = summarize(rep)
    out["jobs"] = n_jobs
    out["sample"] = "first %.0f s of wall time of %s (arrival seed 2024)" % (seconds, label)
    del srv
    torch.cuda.empty_cache()
    return out


def main():
    args = _args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank != 0:
            return 0
        rate, n, el = oracle_wator_rate(None, steps=max(args.steps, 1), warmup=args.warmup)
        import multiprocessing
        line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
                "steps": n, "warmup": args.warmup, "ms_per_step": el * 1e3 / n, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": dict(WORKLOAD),
                "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": "%d wa-tor 2048x2048 steps after %d warm-up steps" % (n, args.warmup)},
                "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch

    if world > 1:
        torch.distributed.init_process_group("nccl")
    r = run_gpu(args, rank, world)
    dev_s, visits, allocfree, e2e_s = r["dev_s"], r["visits"], r["allocfree"], r["e2e_s"]
    if world > 1:
        t = torch.tensor([dev_s, e2e_s], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        n = torch.tensor([visits, allocfree, r["e2e_visits"]], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(n, op=torch.distributed.ReduceOp.SUM)
        dev_s, e2e_s = float(t[0]), float(t[1])
        visits, allocfree, e2e_visits = int(n[0]), int(n[1]), int(n[2])
    else:
        e2e_visits = r["e2e_visits"]
    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0
    peak, peak_kind = _peaks()
    line = {
        "metric": METRIC, "value": visits / dev_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": dict(WORKLOAD, parallelism="replicas" if world > 1 else "single"),
        "alloc_free_per_s": allocfree / dev_s,
        "phase_ms": r["phase_ms"], "clocks": r["clocks"],
        "e2e": {"value": e2e_visits / e2e_s, "unit": UNIT, "h2d_bytes_per_step": r["h2d"] / args.steps,
                "d2h_bytes_per_step": r["d2h"] / args.steps},
        "gpu_launches": 10 * args.steps,
        "roofline": {"bound": "hbm", "achieved": r["f1_gbs"], "peak": peak, "unit": "GB/s",
                     "frac": r["f1_gbs"] / peak, "traffic": None,
                     "kernel": "dsr_doall_kernel<MFishChoose> (fish-choice method kernel)",
                     "algorithmic_bytes_per_launch": r["f1_bytes"], "launch_ms": r["f1_ms"],
                     "peak_source": peak_kind + " hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
                     else "fallback 6.8 TB/s"},
    }
    if not args.no_cpu_baseline:
        rate, n, el = oracle_wator_rate(args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "first %d steps of the same wa-tor 2048x2048 run (%.1f s)" % (n, el)}
    if world == 1 and not args.no_extra:
        # the other halves of the metric: batched vs plain, alloc+free/s, the
        # streaming do-all against the HBM roofline, and the served form
        line["batched"] = bench_batched()
        line["alloc_free_microbench"] = bench_alloc_free()
        line["streaming_doall"] = bench_streaming_doall()
        if args.served_seconds > 0:
            line["served"] = bench_served(args.served_seconds)
            # the same arrival process with jobs small enough to finish inside
            # the bench's budget, so that job latencies exist
            line["served_small"] = bench_served(args.served_seconds, n_jobs=2000, arena_gb=16, lo=64, hi=512,
                                                steps_lo=50, steps_hi=200,
                                                label="a 2,000-job stream with sides in [64, 512] and 50-200 steps")
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
