#!/usr/bin/env python
"""Benchmark of the dsr hot path: one JSON line on rank 0.

Workload: wa-tor on a 2048 x 2048 torus (30% fish, 3% sharks, seed 1), the
plain one-simulation form. A step is one wa-tor step: five parallel do-alls
with device new/delete for births and deaths, i.e. every row of the hot
path. Three of them scan and compact the block list; F2 and S2 run over the
lists of F1 and S1, which create and delete nothing.

  value      do-all object-updates/s (objects visited by method kernels per
             second of device time), inputs resident in HBM;
  e2e        the same metric through the C ABI with the initial grid in
             pinned host memory: host->device copy, heap reset, agent
             creation, the K steps and the device->host read of the final
             state hash all inside the timed region;
  roofline   the method kernel with the largest share of a step: its
             algorithmic bytes (per-object and per-event byte counts of the
             wa-tor rules, see phase_bytes) over its CUDA-event time, both
             summed over the timed steps, against the measured HBM copy
             peak. Times come from events recorded around every scan and
             method kernel inside the timed region; the event counts
             (objects, blocks, moves, births, deaths) from a replay of the
             same steps, checked against the timed window's visit count;
  cpu_baseline  the oracle (single-threaded C++) on the same workload, and
             bounded samples of the other configurations (configs).

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
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="dsr", choices=["dsr", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-extra", action="store_true", help="headline only (no batched/served/microbenchmarks)")
    p.add_argument("--served-seconds", type=float, default=20.0)
    p.add_argument("--leg", choices=sorted(LEGS), help="run one secondary benchmark alone and print its result")
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


def _oracle_instance_rate(args):
    """One batched-workload instance on the oracle (runs in a spawned
    worker): (object-updates, seconds) of `steps` steps after `warmup`."""
    side, seed, warmup, steps = args
    import oracle as Ow
    from paper_1809_07444_gb300 import workloads as WLw
    w = Ow.Wator(side, side, WLw.wator_initial(side, side, seed), seed=seed)
    w.step(warmup)
    upd, t0 = 0, time.perf_counter()
    for _ in range(steps):
        nf, ns = w.counts()
        ev = w.step(1)[0]
        upd += 2 * nf + ns + 2 * (ns - int(ev[3]))
    return upd, time.perf_counter() - t0


def oracle_config_rates():
    """The oracle on the other configurations, each a bounded sample: game
    of life 64x64 (100 generations, one core), n-body 65,536 bodies in FP64
    (one step, rows split over all cores), the batched workload (every
    fourth of the 256 instances, 3 steps each after 3 warm-up steps, one
    spawned process per core), traffic 8192 x 4096 (3 steps after 1 warm-up
    step, one core) and sugarscape 4096 x 4096 (2 steps after 1, one core)."""
    import multiprocessing
    import oracle as O
    from paper_1809_07444_gb300 import workloads as WL

    cores = os.cpu_count() or 1
    out = {}
    g = O.Gol(64, 64, WL.gol_initial(64, 64, 1))
    t0 = time.perf_counter()
    g.step(100)
    out["gol_64"] = {"gens_per_s": 100 / (time.perf_counter() - t0), "cores": 1, "sample": "100 generations"}
    rows, _ = WL.nbody_initial(65536, 1)
    O.set_threads(cores)
    nb = O.NBody(rows)
    t0 = time.perf_counter()
    nb.step(1)
    dt = time.perf_counter() - t0
    O.set_threads(1)
    out["nbody_65536"] = {"s_per_step": dt, "flops": 28.0 * 65536 * 65536 / dt, "cores": cores,
                          "sample": "the first step, FP64", "flop_per_pair": 28}
    c = TRAFFIC_APP
    tr = O.Traffic(c["R"], c["L"], WL.traffic_initial(c["R"], c["L"], SEED, c["density"], c["vmax"]), SEED,
                   vmax=c["vmax"], p=c["p"], alpha=c["alpha"])
    tr.step(1)
    cars = 0
    t0 = time.perf_counter()
    for _ in range(3):
        cars += tr.count()
        tr.step(1)
    dt = time.perf_counter() - t0
    out["traffic"] = {"car_updates_per_s": cars / dt, "cores": 1, "sample": "steps 2-4"}
    del tr
    cap, ag = WL.sugarscape_initial(SUGAR_SIDE, SUGAR_SIDE, SEED)
    sg = O.Sugarscape(SUGAR_SIDE, SUGAR_SIDE, cap, ag, SEED)
    sg.step(1)
    t0 = time.perf_counter()
    sg.step(2)
    dt = time.perf_counter() - t0
    out["sugarscape"] = {"agent_steps_per_s": 2 * len(ag) / dt, "cores": 1, "sample": "steps 2-3"}
    del sg
    sides = [int(s) for s in WL.batched_sides(256, 1)]
    jobs = [(sides[i], 1000 + i, 3, 3) for i in range(0, 256, 4)]
    t0 = time.perf_counter()
    with multiprocessing.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_instance_rate, jobs)
    wall = time.perf_counter() - t0
    upd = sum(u for u, _ in res)
    out["batched"] = {"object_updates_per_s_all_cores": upd / wall,
                      "object_updates_per_s_per_core": upd / sum(t for _, t in res), "cores": cores,
                      "sample": "every fourth of the 256 instances, steps 4-6, one process per core"}
    return out


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
# NVML clocks-event reason bits (nvml.h): power capping, and the slowdowns
# that make a timing run suspect
NVML_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}


def nvml_reason_names(bits):
    """Names of the reasons above that are set in an NVML reason word."""
    return sorted(name for bit, name in NVML_REASONS.items() if bits & bit)


class NvmlSampler:
    """SM clock and clocks-event reasons of one GPU, read through NVML (the
    driver's management library, read-only queries) about every millisecond
    in a thread, so that a timed region of a few milliseconds still gets
    several samples. Raises on __init__ when NVML is not available."""

    def __init__(self, index):
        nv = C.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.nv = nv
        self.h = C.c_void_p()
        if nv.nvmlDeviceGetHandleByIndex_v2(C.c_uint(index), C.byref(self.h)) != 0:
            raise RuntimeError("no NVML device %d" % index)
        self.reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = C.c_uint(0)
        nv.nvmlDeviceGetMaxClockInfo(self.h, C.c_int(1), C.byref(mx))  # NVML_CLOCK_SM = 1
        self.max_mhz = float(mx.value)
        self.samples = []  # (sm MHz, reason bits)
        self.stop = threading.Event()

    def _run(self):
        clk, rs = C.c_uint(0), C.c_ulonglong(0)
        while not self.stop.is_set():
            if self.nv.nvmlDeviceGetClockInfo(self.h, C.c_int(1), C.byref(clk)) == 0 and \
                    self.reasons_fn(self.h, C.byref(rs)) == 0:
                self.samples.append((float(clk.value), int(rs.value)))
            time.sleep(0.0005)

    def start(self):
        self.t = threading.Thread(target=self._run, daemon=True)
        self.t.start()
        t0 = time.perf_counter()
        while not self.samples and time.perf_counter() - t0 < 1.0:  # sampling before the region starts
            time.sleep(0.0005)

    def finish(self):
        self.stop.set()
        self.t.join(timeout=2)


class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.nvml = None

    def __enter__(self):
        try:
            self.nvml = NvmlSampler(self.index)
            self.nvml.start()
            return self
        except Exception:
            self.nvml = None
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
        if self.nvml:
            self.nvml.finish()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.nvml and self.nvml.samples:
            sm = [c for c, _ in self.nvml.samples]
            bits = 0
            for _, r in self.nvml.samples:
                bits |= r
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": self.nvml.max_mhz,
                    "reasons": nvml_reason_names(bits), "samples": len(sm), "source": "nvml, ~1 ms"}
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
                "reasons": sorted(reasons), "samples": len(self.rows), "source": "nvidia-smi, 200 ms"}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
PHASES = ("F1", "F2", "S0", "S1", "S2")
# kernels of one wa-tor step: a scan and a method kernel for F1, S0 and S1; a
# method kernel alone for F2 and S2 (they run over the lists of F1 and S1)
LAUNCHES_PER_STEP = 8
KERNELS = {"F1": "dsr_doall_kernel<MFishChoose>", "F2": "dsr_doall_kernel<MFishMove>",
           "S0": "dsr_doall_kernel<MSharkStarve>", "S1": "dsr_doall_kernel<MSharkChoose>",
           "S2": "dsr_doall_kernel<MSharkMove>"}


def phase_bytes(phase, objs, blocks, moves, births, deaths):
    """Algorithmic bytes of one wa-tor method kernel: what its rules read and
    write per visited object and per event, plus the 12-byte R entry (block id
    and live mask) of every listed block. Fields, grid words, claim words and
    intents are 4 bytes each.

      F1  per fish: x, y, timer read, timer written (16), four neighbour grid
          words (16), intent written (4), claim read-modify-written (8; an
          upper bound, as fish with no empty neighbour claim nothing)   = 44
      F2  per fish: x, y (8), intent (4), claim (4)                      = 16
          per move: target and own grid words written (8), x, y written
          (8), timer read (4), the claim word reset (4)                  = 24
          per birth: timer reset (4), the new fish's three fields (12)   = 16
      S0  per shark: energy read and written                             = 8
          per death: x, y read (8), grid word cleared (4)                = 12
      S1  as F1                                                          = 44
      S2  per shark as F2                                                = 16
          per move: target grid word read and written (8), own grid word
          written (4), x, y written (8), timer read (4), claim reset (4) = 28
          per fish eaten: energy read and written                        = 8
          per birth: timer reset (4), the new shark's four fields (16)   = 20
    """
    per_obj = {"F1": 44, "F2": 16, "S0": 8, "S1": 44, "S2": 16}[phase]
    b = per_obj * objs + 12 * blocks
    if phase == "F2":
        b += 24 * moves + 16 * births
    elif phase == "S0":
        b += 12 * deaths
    elif phase == "S2":
        b += 28 * moves + 8 * deaths + 20 * births
    return b


def replay_phase_counts(lib, k0, seed, warmup, steps, L, flush=None):
    """Event counts of each phase over steps [warmup, warmup + steps) of a
    fresh run of the same simulation (wa-tor is deterministic, so this is the
    timed window's work): objects visited, blocks listed, moves, births and
    deaths, summed per phase. Host synchronisation between phases. Each
    phase's scan and method kernel are also timed with CUDA events
    ("scan_ms", "method_ms", summed), with L2 flushed (`flush`, a buffer
    larger than L2) before every step as in the timed steps."""
    import torch
    from paper_1809_07444_gb300.apps import Wator
    from paper_1809_07444_gb300.heap import _stream_ptr

    w = Wator(W_SIDE, W_SIDE, k0, seed)
    sp = _stream_ptr()
    wh = C.c_void_p(w.handle.value)
    methods = {"F1": (0, L.METHOD_WATOR_F1), "F2": (0, L.METHOD_WATOR_F2), "S0": (1, L.METHOD_WATOR_S0),
               "S1": (1, L.METHOD_WATOR_S1), "S2": (1, L.METHOD_WATOR_S2)}
    w.step(warmup)
    tot = {p: dict(objs=0, blocks=0, moves=0, births=0, deaths=0, scan_ms=0.0, method_ms=0.0) for p in PHASES}
    stream = torch.cuda.current_stream()
    for k in range(steps):
        if flush is not None:
            flush.fill_(k & 0xFF)
        for p in PHASES:
            t, m = methods[p]
            c0 = w.heap.counters()
            a, b, e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
            a.record(stream)
            L.check(lib.dsr_doall_scan(w.heap.handle, t, sp), "dsr_doall_scan")
            b.record(stream)
            torch.cuda.synchronize()
            nblocks = int(w.heap.arena[8:12].cpu().view(torch.int32).item())  # R length in the heap header
            e0.record(stream)
            L.check(lib.dsr_doall_run(w.heap.handle, t, m, C.byref(wh), C.sizeof(wh), sp), "dsr_doall_run")
            e1.record(stream)
            e1.synchronize()
            c1 = w.heap.counters()
            d = tot[p]
            d["scan_ms"] += a.elapsed_time(b)
            d["method_ms"] += e0.elapsed_time(e1)
            d["objs"] += c1["visits"] - c0["visits"]
            d["blocks"] += nblocks
            d["moves"] += c1["app0"] - c0["app0"]
            d["births"] += c1["allocs"] - c0["allocs"]
            d["deaths"] += c1["frees"] - c0["frees"]
    if w.heap.stats()["error_flags"]:
        raise RuntimeError("device error flags in the replay")
    del w
    return tot


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
    seed = replica_seed(rank)
    k0 = WL.wator_initial(W_SIDE, W_SIDE, seed)
    sim = Wator(W_SIDE, W_SIDE, k0, seed)
    stream = torch.cuda.current_stream()
    sp = _stream_ptr(stream)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up, every phase timed: the slowest method kernel is the one the
    # timed steps bracket with events (the roofline kernel); events around
    # every kernel would lengthen the timed steps themselves
    sim.phase_timing(args.warmup)
    for _ in range(args.warmup):
        L.check(lib.dsr_wator_step(sim.handle, 1, sp), "dsr_wator_step")
    warm_ms, _, n_warm = sim.phase_times()
    dominant = max(PHASES, key=lambda p: warm_ms[p]) if n_warm else None
    torch.cuda.synchronize()
    c0 = sim.heap.counters()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sim.phase_timing(args.steps)
    sim.phase_select(PHASES.index(dominant) if dominant else None)
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

    phase_ms, scan_ms, n_rec = sim.phase_times()
    sim.phase_select(None)
    sim.phase_timing(0)
    if n_rec != args.steps:
        raise RuntimeError("phase timing recorded %d of %d steps" % (n_rec, args.steps))
    counts = replay_phase_counts(lib, k0, seed, args.warmup, args.steps, L, flush)
    replay_visits = sum(c["objs"] for c in counts.values())
    if replay_visits != visits:
        raise RuntimeError("replay visited %d objects, the timed window %d" % (replay_visits, visits))
    phases = {}
    for p in PHASES:
        c = dict(counts[p])
        r_scan, r_method = c.pop("scan_ms"), c.pop("method_ms")
        timed = dominant is None or p == dominant
        ms = phase_ms[p] if timed else r_method
        by = phase_bytes(p, **c)
        phases[p] = dict(c, kernel=KERNELS[p], method_ms_per_step=ms / args.steps,
                         scan_ms_per_step=(scan_ms[p] if dominant is None else r_scan) / args.steps,
                         bytes_per_launch=by / args.steps, gbs=by / (ms * 1e-3) / 1e9 if ms > 0 else None,
                         timing="timed steps" if timed else "replay of the timed steps",
                         replay_method_ms_per_step=r_method / args.steps)

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
    e2e_s = time.perf_counter() - t_host0  # host wall clock: ctypes, launches and copies included
    e2e_dev_s = e0.elapsed_time(e1) / 1e3
    lib.dsr_wator_destroy(h2)
    c2 = sim.heap.counters()  # counters restarted at the reset
    hashed = sim.heap.stats()["live_objects"][0]  # objects the final hash do-all visited
    return {
        "dev_s": dev_s, "visits": visits, "allocfree": allocfree, "clocks": clk.summary(),
        "phases": phases, "e2e_s": e2e_s, "e2e_dev_s": e2e_dev_s, "e2e_visits": c2["visits"] - hashed,
        "h2d": k0_host.numel(), "d2h": 16, "stats": st,
    }


# ---------------------------------------------------------------------------
# secondary measurements (rank 0, after the headline)
# ---------------------------------------------------------------------------
def _ev():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


TYPES4 = [[4, 4], [4, 4, 4], [4, 4, 4, 4], [4] * 8]  # capacities 64, 42, 32, 16


def bench_alloc_free(n=1 << 24, n_types=2, reps=2, churn=False):
    """Allocation microbenchmark: n threads each create one object (type by a
    hash of the thread index, among the first n_types of TYPES4), then one
    kernel deletes every object; with churn, a kernel in between where half
    of the threads delete their object and create a replacement. Fresh heap
    each round, L2 flushed before each timed kernel, first round untimed."""
    import torch
    from paper_1809_07444_gb300 import _lib as L
    from paper_1809_07444_gb300.heap import Heap, heap_bytes_for_blocks, _stream_ptr

    caps = [64, 42, 32, 16][:n_types]
    blocks = int(n * sum(1.0 / c for c in caps) / n_types * 1.6) + 4096
    h = Heap(TYPES4, heap_bytes_for_blocks(TYPES4, blocks))
    refs = torch.empty(n, dtype=torch.int64, device="cuda")
    nrep = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ta, tf, tc, replaced = [], [], [], 0
    for r in range(reps + 1):
        h.reset()
        flush.fill_(r)
        a0, a1 = _ev()
        a0.record()
        h.bench_alloc(refs, n_types, 77 + r)
        a1.record()
        if churn:
            nrep.zero_()
            flush.fill_(r + 2)
            c0, c1 = _ev()
            c0.record()
            L.check(h.lib.dsr_bench_churn(h.handle, n, n_types, 1000 + r, C.c_void_p(refs.data_ptr()),
                                          C.c_void_p(nrep.data_ptr()), _stream_ptr()), "dsr_bench_churn")
            c1.record()
        flush.fill_(r + 1)
        f0, f1 = _ev()
        f0.record()
        h.bench_free(refs)
        f1.record()
        torch.cuda.synchronize()
        if r:  # first round warms up
            ta.append(a0.elapsed_time(a1) / 1e3)
            tf.append(f0.elapsed_time(f1) / 1e3)
            if churn:
                tc.append(c0.elapsed_time(c1) / 1e3)
                replaced = int(nrep.item())
    st = h.stats()
    ok = st["error_flags"] == 0 and st["free_blocks"] == st["n_blocks"]
    ma, mf = statistics.median(ta), statistics.median(tf)
    out = {"objects": n, "types": n_types, "allocs_per_s": n / ma, "frees_per_s": n / mf,
           "alloc_free_per_s": 2 * n / (ma + mf), "heap_consistent_after": ok}
    if churn:
        out["churn"] = {"replaced": replaced, "ops_per_s": 2 * replaced / statistics.median(tc),
                        "ms": statistics.median(tc) * 1e3}
    del h, refs, flush
    torch.cuda.empty_cache()
    return out


def bench_atomics(n_words=1 << 24, iters=64):
    """L2 atomic ceiling (no vendor figure): one thread per 64-bit word,
    alternating atomicOr / atomicAnd of one bit on its own word, as
    reductions (results unused) and as dependent atomics (results used)."""
    import torch
    from paper_1809_07444_gb300 import _lib as L
    from paper_1809_07444_gb300.heap import _stream_ptr

    lib = L.load()
    words = torch.zeros(n_words, dtype=torch.int64, device="cuda")
    out = {"words": n_words, "atomics_per_thread": iters}
    for name, ret in (("reductions_per_s", 0), ("dependent_atomics_per_s", 1)):
        ts = []
        for r in range(4):
            a, b = _ev()
            a.record()
            L.check(lib.dsr_bench_atomics(C.c_void_p(words.data_ptr()), n_words, iters, ret, _stream_ptr()),
                    "dsr_bench_atomics")
            b.record()
            b.synchronize()
            if r:
                ts.append(a.elapsed_time(b) * 1e-3)
        out[name] = n_words * iters / statistics.median(ts)
    del words
    return out


def bench_alloc_sweep():
    """M1: 2^24 objects with 1..4 types, 2^26 and 2^28 with 2 types, and the
    50% churn mix at 2^26; beside them the L2 atomic ceiling."""
    rows = [bench_alloc_free(1 << 24, t) for t in (1, 2, 3, 4)]
    rows.append(bench_alloc_free(1 << 26, 2, churn=True))
    rows.append(bench_alloc_free(1 << 28, 2, reps=1))
    return {"rows": rows, "l2": "flushed before each kernel",
            "types": "first n of 4 types with capacities 64, 42, 32, 16", "l2_atomic_ceiling": bench_atomics()}


def bench_streaming_doall(n=1 << 28, fields=4, reps=5):
    """M2: one type with `fields` int32 fields, n objects (>> L2), method
    field f += field f+1 (every field read and written). Timed at full blocks,
    then again after a do-all deleted every fourth object (75% fill)."""
    import torch
    from paper_1809_07444_gb300 import _lib as L
    from paper_1809_07444_gb300.heap import Heap, heap_bytes_for_blocks, _stream_ptr

    types = [[4] * fields]
    h = Heap(types, heap_bytes_for_blocks(types, n // 64 + 1024))
    refs = torch.empty(n, dtype=torch.int64, device="cuda")
    h.bench_alloc(refs, 1, 5)
    del refs
    torch.cuda.synchronize()
    lib, sp = h.lib, _stream_ptr()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    peak, kind = _peaks()
    out = {}
    for fill in ("100%", "75%"):
        if fill == "75%":
            h.parallel_do(0, L.METHOD_DELETE_IF, L.DeleteIfArgs(4, 0))
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
        # algorithmic bytes: every live object's fields read and written
        # once, plus the R entry (12 B) of each listed block
        bytes_method = live * fields * 4 * 2 + alloc_blocks * 12
        t = statistics.median(ms) * 1e-3
        out[fill] = {"objects": live, "method_ms": t * 1e3, "doall_ms": statistics.median(ms_full),
                     "object_updates_per_s": live / t, "achieved_gbs": bytes_method / t / 1e9,
                     "frac": bytes_method / t / 1e9 / peak, "algorithmic_bytes": bytes_method,
                     "fill": live / (alloc_blocks * 64)}
    out.update(fields=fields, peak_gbs=peak, peak_source=kind)
    del h, flush
    torch.cuda.empty_cache()
    return out


def bench_streaming_sweep(n=1 << 28):
    """M2 for K = 2, 4, 8 fields."""
    return {"K%d" % k: bench_streaming_doall(n, k) for k in (2, 4, 8)}


def bench_gol(W=64, gens=100, reps=3):
    """C1: game of life 64 x 64 for 100 generations (three do-alls each);
    latency-bound (the state stays in L2): generations/s and the per-
    generation latency from events around every generation."""
    import torch
    from paper_1809_07444_gb300 import workloads as WL
    from paper_1809_07444_gb300.apps import Gol

    lat, rates = [], []
    for r in range(reps + 1):
        g = Gol(W, W, WL.gol_initial(W, W, 1))
        g.step(1)
        torch.cuda.synchronize()
        evs = [_ev() for _ in range(gens)]
        for k in range(gens):
            evs[k][0].record()
            g.step(1)
            evs[k][1].record()
        torch.cuda.synchronize()
        per = [a.elapsed_time(b) for a, b in evs]
        tot = evs[0][0].elapsed_time(evs[-1][1])
        if r:
            lat.extend(per)
            rates.append(gens / (tot * 1e-3))
        del g
    lat.sort()
    return {"workload": "game of life %dx%d, %d generations" % (W, W, gens), "gens_per_s": statistics.median(rates),
            "gen_ms_p50": lat[len(lat) // 2], "gen_ms_p99": lat[int(len(lat) * 0.99)], "kernels_per_gen": 6,
            "graph": "one graph launch per generation"}


def bench_comparators(steps=50, warmup=5):
    """Section 4 comparators on the bench workload, timed like the headline
    (L2 flushed before every step, CUDA events per step): wa-tor 2048 x 2048
    with no dynamic allocation (agents in per-cell SOA arrays, and in
    per-cell AOS structs; every phase a kernel over all 4.2 M cells), and
    with the BitmapAlloc comparator (per-type object arrays of structs, flat
    bitmaps). All make the same visits as the dsr form, so object-updates/s
    compare."""
    import torch
    from paper_1809_07444_gb300 import workloads as WL
    from paper_1809_07444_gb300.apps import WatorStatic

    from paper_1809_07444_gb300.apps import WatorBitmap

    k0 = WL.wator_initial(W_SIDE, W_SIDE, SEED)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for name, aos in (("static_soa", False), ("static_aos", True), ("bitmap_alloc_aos", None)):
        if aos is None:
            w = WatorBitmap(W_SIDE, W_SIDE, k0, SEED)
            w.visits = lambda w=w: w.heap.counters()["visits"]
        else:
            w = WatorStatic(W_SIDE, W_SIDE, k0, SEED, aos=aos)
        w.step(warmup)
        torch.cuda.synchronize()
        v0 = w.visits()
        evs = [_ev() for _ in range(steps)]
        for k in range(steps):
            flush.fill_(k & 0xFF)
            evs[k][0].record()
            w.step(1)
            evs[k][1].record()
        torch.cuda.synchronize()
        t = sum(a.elapsed_time(b) for a, b in evs) / 1e3
        v = w.visits() - v0
        out[name] = {"ms_per_step": t * 1e3 / steps, "object_updates_per_s": v / t,
                     "launches_per_step": 5 if aos is not None else LAUNCHES_PER_STEP}
        del w
    del flush
    torch.cuda.empty_cache()
    out["workload"] = "wator-2048x2048, steps %d-%d, L2 flushed before every step" % (warmup + 1, warmup + steps)
    return out


TRAFFIC_APP = {"R": 8192, "L": 4096, "density": 0.2, "vmax": 5, "p": 0.25, "alpha": 0.5}


def bench_traffic(steps=30, warmup=3):
    """Traffic (Fig. 6g, Nagel-Schreckenberg) on 8192 open roads of 4096
    cells, 20% occupied (6.7 M cars), L2 flushed before every step, CUDA
    events per step. Algorithmic bytes per step: 21 per car visited (road, x,
    v read; x, v written; the new occupancy mark), 13 per source visited, and
    the occupancy grid read once and cleared once (2 bytes per cell)."""
    import torch
    from paper_1809_07444_gb300 import workloads as WL
    from paper_1809_07444_gb300.apps import Traffic

    c = TRAFFIC_APP
    R, L = c["R"], c["L"]
    w = Traffic(R, L, WL.traffic_initial(R, L, SEED, c["density"], c["vmax"]), SEED, vmax=c["vmax"], p=c["p"],
                alpha=c["alpha"])
    w.step(warmup)
    torch.cuda.synchronize()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ctr0 = w.heap.counters()
    cars0 = w.count()
    evs = [_ev() for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        evs[k][0].record()
        w.step(1)
        evs[k][1].record()
    torch.cuda.synchronize()
    t = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    ctr1 = w.heap.counters()
    visits = ctr1["visits"] - ctr0["visits"]
    src_visits = R * steps
    car_visits = visits - src_visits
    vsum = ctr1["app3"] - ctr0["app3"]
    alg = car_visits * 21 + src_visits * 13 + 2 * R * L * steps
    peak, peak_kind = _peaks()
    del w, flush
    torch.cuda.empty_cache()
    return {"workload": "traffic %d roads x %d cells, %.0f%% occupied, vmax %d, p %.2f, alpha %.2f, steps %d-%d, "
                        "L2 flushed before every step" % (R, L, 100 * c["density"], c["vmax"], c["p"], c["alpha"],
                                                          warmup + 1, warmup + steps),
            "ms_per_step": t * 1e3 / steps, "car_updates_per_s": car_visits / t, "object_updates_per_s": visits / t,
            "cars_at_start": cars0, "flow_per_cell": vsum / (R * L * steps),
            "entered": ctr1["app0"] - ctr0["app0"], "left": ctr1["app1"] - ctr0["app1"],
            "algorithmic_gbs": alg / t / 1e9, "hbm_frac": alg / t / 1e9 / peak, "peak_gbs": peak,
            "peak_kind": peak_kind, "launches_per_step": 4, "memsets_per_step": 1}


SUGAR_SIDE = 4096


def bench_sugarscape(steps=30, warmup=3):
    """Sugarscape (Fig. 6f) on a 4096 x 4096 torus, 10% of the cells holding
    an agent (1.68 M agents), L2 flushed before every step, CUDA events per
    step. Object-updates: four do-alls visit every agent each step.
    Algorithmic bytes per agent per step: A1 reads x, y, vision (12) and the
    cells in sight (occupancy, capacity, harvest step: 6 bytes a cell, 4 x
    vision cells, vision 3.5 on average) and writes the intent (4); A2 reads
    six fields and the intent (28), writes sugar, age, dead (12) and its
    cell's harvest step (capacity and step read, step written: 9); A3 and A4
    read the dead flag (4 each)."""
    import torch
    from paper_1809_07444_gb300 import workloads as WL
    from paper_1809_07444_gb300.apps import Sugarscape

    cap, agents = WL.sugarscape_initial(SUGAR_SIDE, SUGAR_SIDE, SEED)
    g = Sugarscape(SUGAR_SIDE, SUGAR_SIDE, cap, agents, SEED)
    g.step(warmup)
    torch.cuda.synchronize()
    ev0 = g.events()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    evs = [_ev() for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        evs[k][0].record()
        g.step(1)
        evs[k][1].record()
    torch.cuda.synchronize()
    t = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    ev1 = g.events()
    n = len(agents)
    per_agent = (12 + 6 * 4 * 3.5 + 4) + (28 + 12 + 9) + 4 + 4
    alg = n * per_agent * steps
    peak, peak_kind = _peaks()
    del g, flush
    torch.cuda.empty_cache()
    d = [b - a for a, b in zip(ev0, ev1)]
    return {"workload": "sugarscape %dx%d, %d agents, steps %d-%d, L2 flushed before every step"
                        % (SUGAR_SIDE, SUGAR_SIDE, n, warmup + 1, warmup + steps),
            "ms_per_step": t * 1e3 / steps, "agent_steps_per_s": n * steps / t,
            "object_updates_per_s": 4 * n * steps / t, "moves": d[0], "deaths": d[1] + d[2],
            "algorithmic_gbs": alg / t / 1e9, "hbm_frac": alg / t / 1e9 / peak, "peak_gbs": peak,
            "peak_kind": peak_kind, "launches_per_step": 5}


def bench_space(heap_bytes=32 << 20, steps=100):
    """Fig. 8: the largest wa-tor torus a 32 MB heap runs for 100 steps
    without running out of memory, per tuning, with the peak bytes of live
    object data as a fraction of the heap."""
    from paper_1809_07444_gb300 import space

    t0 = time.perf_counter()
    out = space.experiment(heap_bytes, steps)
    out["search_s"] = time.perf_counter() - t0
    return out


def bench_nbody(n=65536, steps=5):
    """C3: n-body with merging, 65,536 bodies (FP32-pair state, FP64 update and
    merges), in both pair-force modes: FP32 pairs (FP64 for pairs within
    r_near) and FP64 pairs. FLOPs counted as 20 per pair for the all-pairs
    force (softened inverse-cube, three FMAs into the acceleration; the
    near field and the merge-partner search only visit neighbouring cells
    and are not counted), against the FP32 FMA ceiling measured by
    dsr_bench_fma."""
    import torch
    from paper_1809_07444_gb300 import _lib as L
    from paper_1809_07444_gb300 import workloads as WL
    from paper_1809_07444_gb300.apps import NBody
    from paper_1809_07444_gb300.heap import _stream_ptr

    rows, _ = WL.nbody_initial(n, 1)
    out = {"workload": "n-body %d bodies, steps 3-%d" % (n, 2 + steps), "bound": "alu", "flop_per_pair": 20}
    for mode in ("fp32", "fp64"):
        nb = NBody(rows, pairs=mode)
        nb.step(2)
        torch.cuda.synchronize()
        live0 = nb.heap.stats()["live_objects"][0]
        e0, e1 = _ev()
        e0.record()
        nb.step(steps)
        e1.record()
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / steps
        out[mode + "_pairs"] = {"ms_per_step": t * 1e3, "bodies": live0, "tflops": 20.0 * live0 * live0 / t / 1e12,
                                "near_pairs_last_step": nb.near_pairs(), "r_near": nb.params.r_near}
        del nb
        torch.cuda.empty_cache()
    lib = L.load()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ctas, iters = sms * 8, 1 << 16
    out_buf = torch.empty(ctas * 256, dtype=torch.float32, device="cuda")
    fl = []
    for r in range(4):
        a, b = _ev()
        a.record()
        L.check(lib.dsr_bench_fma(C.c_void_p(out_buf.data_ptr()), ctas, iters, _stream_ptr()), "dsr_bench_fma")
        b.record()
        b.synchronize()
        if r:
            fl.append(ctas * 256 * 8 * iters * 2 / (a.elapsed_time(b) * 1e-3))
    peak = statistics.median(fl)
    out["fp32_fma_peak_tflops"] = peak / 1e12
    f32 = out["fp32_pairs"]
    out["ms_per_step"] = f32["ms_per_step"]
    out["frac_of_fma_peak"] = f32["tflops"] * 1e12 / peak
    return out


def bench_batched_fixed(n_inst=256, steps=20, warmup=3):
    """The batched workload with the default tuning (256 threads, 64-slot
    blocks, fan-out 64) and nothing else: no autotuning, no one-by-one
    comparison. The short case for profiling the batched step."""
    import torch
    from paper_1809_07444_gb300 import workloads as WL
    from paper_1809_07444_gb300.apps import WatorBatch

    sides = [int(s) for s in WL.batched_sides(n_inst, 1)]
    need = sum(WatorBatch.blocks_for(s, s) * 1100 + s * s * 24 for s in sides)
    b = WatorBatch(need + (256 << 20), max_instances=n_inst)
    slots = [b.add(s, s, WL.wator_initial(s, s, 1000 + i), 1000 + i) for i, s in enumerate(sides)]
    b.step(warmup)
    torch.cuda.synchronize()
    v0 = sum(b.heap(x).counters()["visits"] for x in slots)
    e0, e1 = _ev()
    e0.record()
    b.step(steps)
    e1.record()
    e1.synchronize()
    v1 = sum(b.heap(x).counters()["visits"] for x in slots)
    t = e0.elapsed_time(e1) / 1e3
    return {"workload": "wator-batched-%d (sides log-uniform [64, 1024], seeds 1000+i), default tuning" % n_inst,
            "steps": steps, "warmup": warmup, "ms_per_step": t * 1e3 / steps, "object_updates_per_s": (v1 - v0) / t}


def bench_batched(n_inst=256, steps=20, one_by_one_steps=3):
    """The batched workload (256 wa-tor instances, sides log-uniform in
    [64, 1024]) advanced by graph-captured group steps, against the same
    instances stepped one by one in the plain form."""
    import torch
    from paper_1809_07444_gb300 import workloads as WL
    from paper_1809_07444_gb300.apps import Wator, WatorBatch

    from paper_1809_07444_gb300 import autotune as AT

    sides = [int(s) for s in WL.batched_sides(n_inst, 1)]
    # autotune threads / cap_min / fan-out on every fourth instance
    sub = list(range(0, n_inst, 4))
    t0 = time.perf_counter()
    tun, tun_v, table = AT.tuned("%s/wator-batched-%d" % (torch.cuda.get_device_name(), n_inst),
                                 AT.wator_batch_measure([sides[i] for i in sub], [1000 + i for i in sub]),
                                 refresh=True)
    tune_s = time.perf_counter() - t0
    need = sum(WatorBatch.blocks_for(s, s) * 1100 + s * s * 24 for s in sides)
    b = WatorBatch(need + (256 << 20), max_instances=n_inst, tuning=tun)
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
                                                       "launches_per_step": LAUNCHES_PER_STEP * n_inst},
            "speedup_vs_one_by_one": vb / vp if vp else None, "launches_per_step": LAUNCHES_PER_STEP, "graph": True,
            "tuning": tun, "tuning_s": tune_s,
            "tuning_table": {",".join(str(x) for x in k): v for k, v in (table or {}).items()},
            "tuning_sample": "every fourth instance (%d), 5 timed steps per setting" % len(sub)}


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


# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant
# kernel on this workload, mean over the timed launches of one capture, with
# the (steps, warmup) window it was taken on. The bench reports it only when
# it runs that window (the population, hence the bytes of a launch, changes
# from step to step); a kernel changed since its capture has no entry.
TRAFFIC = {"F2": {"bytes": 68276505, "steps": 20, "warmup": 5, "cache_control": "none",
                  "source": "profiles/wator2048_fish_move_traffic.md"}}


def roofline(phases, peak, peak_kind, steps, warmup):
    """HBM roofline of the method kernel with the largest share of the step."""
    timed = [q for q in PHASES if phases[q].get("timing", "timed steps") == "timed steps"]
    p = max(timed or PHASES, key=lambda q: phases[q]["method_ms_per_step"])
    ph = phases[p]
    achieved = ph["gbs"]
    cap = TRAFFIC.get(p)
    same_window = cap is not None and (cap["steps"], cap["warmup"]) == (steps, warmup)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
            "traffic": cap["bytes"] if same_window else None,
            "traffic_window": ({"steps": cap["steps"], "warmup": cap["warmup"], "source": cap["source"],
                                "cache_control": cap.get("cache_control")}
                               if cap is not None else None),
            "kernel": ph["kernel"], "phase": p,
            "algorithmic_bytes_per_launch": ph["bytes_per_launch"], "launch_ms": ph["method_ms_per_step"],
            "timing": "CUDA events on the launching stream around every launch of this kernel in the timed steps",
            "peak_source": ("measured hbm_gbs" if peak_kind == "measured" else "fallback 6.8 TB/s")}


NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal


def batched_hbm_estimate(line, peak):
    """Algorithmic HBM bandwidth of the batched step, estimated: the batched
    form runs the same five phases over instances of the same rules, so its
    bytes per object-update are taken from the plain run's per-phase byte
    counts (summed over the phases of a step) divided by the plain run's
    object-updates per step."""
    bytes_step = sum(ph["bytes_per_launch"] for ph in line["phases"].values())
    visits_step = line["value"] * line["ms_per_step"] / 1e3
    per_update = bytes_step / visits_step
    gbs = line["batched"]["object_updates_per_s"] * per_update / 1e9
    return {"algorithmic_gbs": gbs, "bytes_per_object_update": per_update, "frac": gbs / peak,
            "frac_of_nominal": gbs / NOMINAL_HBM_GBS,
            "method": "plain run's algorithmic bytes per object-update x batched object-updates/s"}


def summary(line):
    """The headline figures of every leg in a few hundred characters: the
    plain and batched forms side by side (the metric's "batched vs plain"),
    allocation, the HBM roofline fractions, n-body and the served form."""
    def g(d, *keys):
        for k in keys:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d

    def r3(x):
        return float("%.4g" % x) if isinstance(x, (int, float)) else x

    out = {"plain_object_updates_per_s": r3(line["value"]), "plain_ms_per_step": r3(line["ms_per_step"]),
           "e2e_object_updates_per_s": r3(g(line, "e2e", "value")),
           "dominant_kernel_frac_of_hbm": r3(g(line, "roofline", "frac"))}
    b = line.get("batched")
    if b:
        out["batched_object_updates_per_s"] = r3(b["object_updates_per_s"])
        out["batched_vs_plain"] = r3(b["object_updates_per_s"] / line["value"])
        out["batched_vs_one_by_one"] = r3(b.get("speedup_vs_one_by_one"))
        out["batched_frac_of_hbm_est"] = r3(g(b, "hbm_est", "frac"))
    a = g(line, "alloc_free_microbench", "rows")
    if a:
        two = [x for x in a if x["types"] == 2 and x["objects"] == 1 << 24]
        if two:
            out["allocs_per_s"] = r3(two[0]["allocs_per_s"])
            out["frees_per_s"] = r3(two[0]["frees_per_s"])
    st = line.get("streaming_doall")
    if st:
        out["streaming_frac_of_hbm_100pct_fill"] = {k: r3(g(v, "100%", "frac")) for k, v in st.items()}
    nb = line.get("nbody_65536")
    if nb:
        out["nbody_ms_per_step"] = {k: r3(g(nb, k + "_pairs", "ms_per_step")) for k in ("fp32", "fp64")}
    for k in ("served", "served_small"):
        sv = line.get(k)
        if sv:
            out[k] = {q: r3(sv.get(q)) for q in ("jobs_done", "step_ms_p50", "step_ms_p99", "step_ms_per_mcell_p50",
                                                  "step_ms_per_mcell_p99", "job_s_p50", "job_s_p99",
                                                  "admit_ms_per_job_p50", "admit_ms_per_job_p99")}
    return out


def combine_ranks(times, counts, world, device):
    """Whole-job figures over the ranks of a replica run: the slowest rank's
    times (max) and the summed counts. One process per GPU, no exchange
    inside the timed region: this runs after it."""
    if world <= 1:
        return list(times), list(counts)
    import torch

    t = torch.tensor(times, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    n = torch.tensor(counts, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(n, op=torch.distributed.ReduceOp.SUM)
    return [float(x) for x in t.tolist()], [int(x) for x in n.tolist()]


def replica_seed(rank):
    """Each rank runs its own wa-tor replica from seed SEED + rank."""
    return SEED + rank


LEGS = {
    "batched": lambda a: bench_batched(),
    # the batched step alone at the default tuning: the case profiled under ncu
    "batched_fixed": lambda a: bench_batched_fixed(),
    "alloc": lambda a: bench_alloc_sweep(),
    # one small allocation round (2^20 objects, 2 types) after one untimed
    # round: the case profiled under ncu
    "alloc_small": lambda a: bench_alloc_free(1 << 20, 2, reps=1),
    "streaming": lambda a: bench_streaming_sweep(),
    "gol": lambda a: bench_gol(),
    "space": lambda a: bench_space(),
    "comparators": lambda a: bench_comparators(),
    "nbody": lambda a: bench_nbody(),
    "traffic": lambda a: bench_traffic(),
    "sugarscape": lambda a: bench_sugarscape(),
    "served": lambda a: bench_served(a.served_seconds),
}


def main():
    args = _args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.leg:
        print(json.dumps({"leg": args.leg, "result": LEGS[args.leg](args)}))
        return 0

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
    (dev_s, e2e_s), (visits, allocfree, e2e_visits) = combine_ranks(
        [r["dev_s"], r["e2e_s"]], [r["visits"], r["allocfree"], r["e2e_visits"]], world, "cuda")
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
        "phases": r["phases"], "clocks": r["clocks"],
        "e2e": {"value": e2e_visits / e2e_s, "unit": UNIT, "h2d_bytes_per_step": r["h2d"] / args.steps,
                "d2h_bytes_per_step": r["d2h"] / args.steps, "timing": "host wall clock around the C-ABI calls",
                "device_s": r["e2e_dev_s"], "host_s": e2e_s},
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
        "roofline": roofline(r["phases"], peak, peak_kind, args.steps, args.warmup),
    }
    if not args.no_cpu_baseline:
        rate, n, el = oracle_wator_rate(args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "first %d steps of the same wa-tor 2048x2048 run (%.1f s)" % (n, el)}
        if world == 1 and not args.no_extra:
            line["cpu_baseline"]["configs"] = oracle_config_rates()
    if world == 1 and not args.no_extra:
        # the other halves of the metric: batched vs plain, alloc+free/s, the
        # streaming do-all against the HBM roofline, and the served form
        line["batched"] = bench_batched()
        line["batched"]["hbm_est"] = batched_hbm_estimate(line, peak)
        line["alloc_free_microbench"] = bench_alloc_sweep()
        line["streaming_doall"] = bench_streaming_sweep()
        line["gol_64"] = bench_gol()
        line["space_efficiency"] = bench_space()
        line["comparators"] = bench_comparators()
        line["nbody_65536"] = bench_nbody()
        line["traffic"] = bench_traffic()
        line["sugarscape"] = bench_sugarscape()
        if args.served_seconds > 0:
            line["served"] = bench_served(args.served_seconds)
            # the same arrival process with jobs small enough to finish within
            # the served time window, so that job latencies exist
            line["served_small"] = bench_served(args.served_seconds, n_jobs=2000, arena_gb=16, lo=64, hi=512,
                                                steps_lo=50, steps_hi=200,
                                                label="a 2,000-job stream with sides in [64, 512] and 50-200 steps")
    line["summary"] = summary(line)  # last key: the end of the line is what a log tail keeps
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
