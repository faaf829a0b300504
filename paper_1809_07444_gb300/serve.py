"""Serving: continuous batching of game-of-life and wa-tor jobs on one GPU.

Jobs arrive over time (a Poisson stream), each with its application, grid
side, step count and seed. Both applications draw on one device arena (a
wa-tor batch and a game-of-life batch sharing its free bytes). A job is
admitted as soon as its heap and workspace fit in the arena's free bytes
(first fit; jobs that do not fit wait, later smaller jobs may pass them).
Admitted jobs stay resident on the device and advance together: one tick is
one batched step of every resident wa-tor job and one batched generation of
every resident game-of-life job (group do-alls replayed from a CUDA graph).
A job that has done its steps leaves at the tick boundary: its final state
hash is read and its bytes are returned, so the next waiting job can start
on the following tick.

Per tick the report separates the device time of the batched step
(step_ms, CUDA events around the graph replays alone) from the host time
spent changing the resident set: admitting jobs (their initial state copied
in and created on the device) and re-capturing the step graphs when the set
changed (admit_ms), and retiring finished jobs (retire_ms).

Host code here only schedules (admission, retirement, bookkeeping); every
step runs in libdsr.so.
"""
import collections
import concurrent.futures as cf
import time

import numpy as np
import torch

from . import workloads as WL
from .apps import GolBatch, WatorBatch

WATOR, GOL = 1, 0


class Server:
    def __init__(self, arena_bytes=64 << 30, max_jobs=4096, tuning=None):
        self.wb = WatorBatch(int(arena_bytes) // 1024 * 1024, max_instances=max_jobs, tuning=tuning)
        self.gb = GolBatch(share=self.wb, max_instances=max_jobs, tuning=tuning)
        self.stream = torch.cuda.current_stream()

    def free_bytes(self):
        """(free bytes, largest free range) of the shared arena."""
        return self.wb.free_bytes()

    @staticmethod
    def _initial(job):
        side, seed = int(job["side"]), int(job["seed"])
        if job["app"] == WATOR:
            return WL.wator_initial(side, side, seed)
        return WL.gol_initial(side, side, seed)

    def _admit(self, job, start):
        side, seed = int(job["side"]), int(job["seed"])
        if job["app"] == WATOR:
            return self.wb.add(side, side, start, seed)
        return self.gb.add(side, side, start)

    def _batch(self, app):
        return self.wb if app == WATOR else self.gb

    def run(self, jobs, time_limit=None, realtime=True, max_admit_per_tick=64, keep_hashes=True, prefetch=64,
            workers=8):
        """Serve `jobs` (a list of dicts with id, arrival, app, side, steps, seed).

        Returns a report: per completed job its arrival, admission, completion
        (seconds since start), ticks and final state hashes; per tick its
        device time; the objects visited; and jobs left unfinished when
        `time_limit` (seconds of wall time) ran out. With realtime=False,
        arrivals are not waited for (every job counts as arrived at start).

        Initial states are generated on the host by a pool of `workers`
        threads, up to `prefetch` jobs ahead in arrival order, while the
        device runs ticks; a waiting job is admitted once its state is ready.
        """
        order = sorted(jobs, key=lambda j: j["arrival"])
        pending = collections.deque(order)
        waiting = collections.deque()
        pool = cf.ThreadPoolExecutor(max_workers=workers)
        starts = {}  # job id -> future of its initial state
        ahead = 0  # jobs of `order` submitted to the pool

        def top_up():
            nonlocal ahead
            while ahead < len(order) and len(starts) < prefetch:
                j = order[ahead]
                starts[j["id"]] = pool.submit(self._initial, j)
                ahead += 1
        resident = {}  # (app, slot) -> [job, steps_left, admitted_at]
        done = []
        ticks = []  # (start event, end event, resident count, resident cells)
        admit_ms, retire_ms = [], []  # host time of ticks that changed the resident set
        admit_n = []  # jobs admitted in those ticks
        cells = 0  # cells of the resident jobs
        t0 = time.perf_counter()
        visits = 0

        def now():
            return time.perf_counter() - t0

        while pending or waiting or resident:
            t = now()
            if time_limit is not None and t > time_limit:
                break
            top_up()
            while pending and (not realtime or pending[0]["arrival"] <= t):
                waiting.append(pending.popleft())
            # admission: first fit in arrival order among jobs whose initial
            # state is ready, bounded per tick
            t_adm = time.perf_counter()
            admitted = 0
            kept = collections.deque()
            while waiting and admitted < max_admit_per_tick:
                job = waiting.popleft()
                fut = starts.get(job["id"])
                if fut is None or not fut.done():
                    kept.append(job)
                    continue
                slot = self._admit(job, fut.result())
                if slot is None:
                    kept.append(job)
                    continue
                del starts[job["id"]]
                resident[(job["app"], slot)] = [job, int(job["steps"]), now()]
                cells += int(job["side"]) ** 2
                admitted += 1
            kept.extend(waiting)
            waiting = kept
            if not resident:
                if pending and realtime:
                    time.sleep(max(0.0, min(pending[0]["arrival"] - now(), 0.05)))
                elif waiting:
                    time.sleep(0.001)  # initial states still being generated
                continue
            # re-capture the step graphs now if the resident set changed, so
            # that the tick's events time the replays alone
            if self.wb.inst:
                self.wb.prepare()
            if self.gb.inst:
                self.gb.prepare()
            if admitted:
                self.stream.synchronize()  # the admitted jobs' initial states are created
                admit_ms.append((time.perf_counter() - t_adm) * 1e3)
                admit_n.append(admitted)
            # one tick: a batched step of each application that has jobs
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            if self.wb.inst:
                self.wb.step(1)
            if self.gb.inst:
                self.gb.step(1)
            b.record(self.stream)
            ticks.append((a, b, len(resident), cells))
            finished = []
            for key, rec in resident.items():
                rec[1] -= 1
                if rec[1] == 0:
                    finished.append(key)
            if finished:
                b.synchronize()
                t_done = now()
                t_ret = time.perf_counter()
                for key in finished:
                    app, slot = key
                    job, _, t_adm = resident.pop(key)
                    cells -= int(job["side"]) ** 2
                    batch = self._batch(app)
                    heap = batch.heap(slot)
                    visits += heap.counters()["visits"]
                    h = batch.hash(slot) if keep_hashes else None
                    batch.remove(slot)
                    done.append({"id": job["id"], "app": app, "side": int(job["side"]), "steps": int(job["steps"]),
                                 "seed": int(job["seed"]), "arrival": float(job["arrival"]), "admitted": t_adm,
                                 "completed": t_done, "hash": h})
                retire_ms.append((time.perf_counter() - t_ret) * 1e3)
        pool.shutdown(wait=False, cancel_futures=True)
        torch.cuda.synchronize()
        wall = now()
        step_ms = [x.elapsed_time(y) for x, y, _, _ in ticks]
        for key, rec in resident.items():  # count the work of jobs still resident
            visits += self._batch(key[0]).heap(key[1]).counters()["visits"]
        return {"done": done, "step_ms": step_ms, "resident": [k for _, _, k, _ in ticks],
                "resident_cells": [c for _, _, _, c in ticks], "admit_ms": admit_ms, "admit_n": admit_n,
                "retire_ms": retire_ms, "wall_s": wall, "visits": visits,
                "unfinished": len(resident) + len(waiting) + len(pending)}


def summarize(report):
    """p50/p99 per-step (device) and per-job latency, the host time of
    admissions and retirements, throughput."""
    def pct(xs, q):
        return float(np.percentile(np.array(xs), q)) if len(xs) else 0.0

    lat = [d["completed"] - d["arrival"] for d in report["done"]]
    # device time per million resident cells: a tick's time grows with the
    # cells resident, so raw tick percentiles mix load with stalls; per cell,
    # a p99 far above the p50 points at stalls
    per_cell = [ms / (c / 1e6) for ms, c in zip(report["step_ms"], report.get("resident_cells", [])) if c]
    per_job = [ms / n for ms, n in zip(report.get("admit_ms", []), report.get("admit_n", [])) if n]
    return {
        "jobs_done": len(report["done"]), "jobs_unfinished": report["unfinished"], "ticks": len(report["step_ms"]),
        "step_ms_p50": pct(report["step_ms"], 50), "step_ms_p99": pct(report["step_ms"], 99),
        "job_s_p50": pct(lat, 50), "job_s_p99": pct(lat, 99),
        "admit_ms_p50": pct(report.get("admit_ms", []), 50), "admit_ms_p99": pct(report.get("admit_ms", []), 99),
        "retire_ms_p50": pct(report.get("retire_ms", []), 50),
        "retire_ms_p99": pct(report.get("retire_ms", []), 99),
        "resident_p50": pct(report.get("resident", []), 50), "resident_max": max(report.get("resident", [0]) or [0]),
        "step_ms_per_mcell_p50": pct(per_cell, 50), "step_ms_per_mcell_p99": pct(per_cell, 99),
        "admit_ms_per_job_p50": pct(per_job, 50), "admit_ms_per_job_p99": pct(per_job, 99),
        "object_updates_per_s": report["visits"] / report["wall_s"] if report["wall_s"] else 0.0,
        "wall_s": report["wall_s"],
    }
