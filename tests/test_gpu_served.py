"""Served form on the GPU: jobs admitted by free bytes and stepped together are each bit-exact vs the oracle,
and a job's result is the same alone as in the mix."""
import numpy as np
import pytest

import oracle as O
from paper_1809_07444_gb300 import workloads as WL
from paper_1809_07444_gb300.serve import GOL, WATOR, Server, summarize

pytestmark = pytest.mark.gpu


def _jobs(n, seed, lo=16, hi=128, steps_lo=5, steps_hi=40):
    s = WL.served_jobs(n, seed, rate=5000.0, lo=lo, hi=hi, steps_lo=steps_lo, steps_hi=steps_hi)
    return [{"id": i, "arrival": float(s["arrival"][i]), "app": int(s["app"][i]), "side": int(s["side"][i]),
             "steps": int(s["steps"][i]), "seed": int(s["seed"][i])} for i in range(n)]


def _oracle_hash(job):
    side, seed, steps = job["side"], job["seed"], job["steps"]
    if job["app"] == WATOR:
        w = O.Wator(side, side, WL.wator_initial(side, side, seed), seed=seed)
        w.step(steps)
        return w.hash()
    g = O.Gol(side, side, WL.gol_initial(side, side, seed))
    g.step(steps)
    return g.hash()


def test_served_jobs_match_oracle_and_queue_for_memory():
    jobs = _jobs(30, 3)
    # small arenas: not every job fits at once, so jobs wait for others to leave
    srv = Server(arena_bytes=6 << 20, max_jobs=64)
    rep = srv.run(jobs, realtime=False)
    assert rep["unfinished"] == 0 and len(rep["done"]) == len(jobs)
    waited = [d for d in rep["done"] if d["admitted"] > 0.0 and d["admitted"] > min(x["completed"] for x in rep["done"])]
    assert waited, "expected some jobs to be admitted only after others completed"
    for d in rep["done"]:
        assert tuple(d["hash"]) == _oracle_hash(d), "job %d (app %d side %d)" % (d["id"], d["app"], d["side"])
    s = summarize(rep)
    assert s["jobs_done"] == 30 and s["step_ms_p99"] >= s["step_ms_p50"] > 0


def test_one_arena_serves_either_application():
    # the two applications draw on one pool of bytes: game-of-life instances
    # alone fill most of the arena, and the bytes they return on leaving are
    # what a wa-tor instance is then admitted into
    srv = Server(arena_bytes=96 << 20, max_jobs=256)
    total = srv.free_bytes()[0]
    slots = []
    while True:
        slot = srv.gb.add(128, 128, WL.gol_initial(128, 128, len(slots)))
        if slot is None:
            break
        slots.append(slot)
    assert len(slots) > 4
    assert total - srv.free_bytes()[0] > 0.8 * total
    k0 = WL.wator_initial(256, 256, 1)
    assert srv.wb.add(256, 256, k0, 1) is None
    for slot in slots:
        srv.gb.remove(slot)
    assert srv.free_bytes()[0] == total
    w = srv.wb.add(256, 256, k0, 1)
    assert w is not None
    ref = O.Wator(256, 256, k0, seed=1)
    srv.wb.step(5)
    ref.step(5)
    assert srv.wb.hash(w) == ref.hash()


def test_tick_report_separates_device_step_and_host_admission():
    jobs = _jobs(20, 11)
    rep = Server(arena_bytes=64 << 20, max_jobs=64).run(jobs, realtime=False)
    s = summarize(rep)
    assert s["jobs_done"] == 20 and len(rep["admit_ms"]) >= 1 and len(rep["retire_ms"]) >= 1
    assert s["admit_ms_p99"] >= s["admit_ms_p50"] > 0 and s["step_ms_p50"] > 0
    assert len(rep["resident"]) == s["ticks"] and s["resident_max"] >= 1


def test_job_result_alone_equals_result_in_mix():
    jobs = _jobs(12, 5)
    target = dict(jobs[7])
    alone = Server(arena_bytes=32 << 20, max_jobs=8).run([dict(target, arrival=0.0)], realtime=False)
    mix = Server(arena_bytes=32 << 20, max_jobs=32).run(jobs, realtime=False)
    h_alone = alone["done"][0]["hash"]
    h_mix = [d["hash"] for d in mix["done"] if d["id"] == target["id"]][0]
    assert h_alone == h_mix == _oracle_hash(target)


def test_poisson_arrivals_in_real_time():
    # arrivals spread over ~30 ms of wall time; every job still completes and matches
    jobs = _jobs(16, 9, steps_hi=20)
    srv = Server(arena_bytes=64 << 20, max_jobs=64)
    rep = srv.run(jobs, realtime=True)
    assert rep["unfinished"] == 0
    for d in rep["done"]:
        assert d["admitted"] >= d["arrival"] - 1e-3
        assert tuple(d["hash"]) == _oracle_hash(d)


def _oracle_hash_job(job):
    # runs in a spawned worker process
    import oracle as O2
    from paper_1809_07444_gb300 import workloads as WL2
    side, seed, steps = job["side"], job["seed"], job["steps"]
    if job["app"] == WATOR:
        w = O2.Wator(side, side, WL2.wator_initial(side, side, seed), seed=seed)
        w.step(steps)
        return job["id"], w.hash()
    g = O2.Gol(side, side, WL2.gol_initial(side, side, seed))
    g.step(steps)
    return job["id"], g.hash()


def _stratified_sample(s, edges=(128, 256, 512, 1024, 2048, 4097), first=40, max_cell_steps=3e9):
    """Jobs of the configured stream, stratified by application and side bin:
    per (app, bin), among the first `first` jobs of the bin whose oracle run
    costs at most `max_cell_steps` cell-steps (a bound on the test's time),
    the first one, the one with the fewest and the one with the most steps."""
    picked = []
    n = len(s["arrival"])
    for app in (GOL, WATOR):
        for lo, hi in zip(edges[:-1], edges[1:]):
            idx = [i for i in range(n) if s["app"][i] == app and lo <= s["side"][i] < hi
                   and int(s["side"][i]) ** 2 * int(s["steps"][i]) <= max_cell_steps][:first]
            assert idx, (app, lo, hi)
            steps = [int(s["steps"][i]) for i in idx]
            for i in {idx[0], idx[int(np.argmin(steps))], idx[int(np.argmax(steps))]}:
                picked.append(i)
    return sorted(set(picked))


def test_configured_stream_stratified_sample_matches_oracle():
    # The served workload's own stream (Poisson 200 jobs/s, 10,000 jobs, sides
    # log-uniform in [128, 4096], 50-1000 steps): a stratified sample of its
    # jobs at their configured sizes and step counts, served together, each
    # final state hash against its own oracle run; the largest wa-tor job of
    # the sample also alone, with the same result.
    import multiprocessing as mp
    import os

    s = WL.served_jobs(10000, 2024)
    ids = _stratified_sample(s)
    assert len(ids) >= 24
    jobs = [{"id": int(i), "arrival": 0.0, "app": int(s["app"][i]), "side": int(s["side"][i]),
             "steps": int(s["steps"][i]), "seed": int(s["seed"][i])} for i in ids]
    assert max(j["side"] for j in jobs) >= 3000 and max(j["steps"] for j in jobs) >= 950
    assert min(j["side"] for j in jobs) < 256 and min(j["steps"] for j in jobs) <= 200
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(jobs), os.cpu_count() or 4)) as pool:
        # the largest jobs first, so that the pool's tail is short
        pending = pool.map_async(_oracle_hash_job, sorted(jobs, key=lambda j: -j["side"] ** 2 * j["steps"]), chunksize=1)
        mix = Server(arena_bytes=48 << 30, max_jobs=64).run(jobs, realtime=False)
        big = max((j for j in jobs if j["app"] == WATOR), key=lambda j: j["side"])
        alone = Server(arena_bytes=8 << 30, max_jobs=4).run([dict(big)], realtime=False)
        want = dict(pending.get())
    assert mix["unfinished"] == 0 and len(mix["done"]) == len(jobs)
    for d in mix["done"]:
        assert tuple(d["hash"]) == tuple(want[d["id"]]), "job %d (app %d side %d steps %d)" % (
            d["id"], d["app"], d["side"], d["steps"])
    assert tuple(alone["done"][0]["hash"]) == tuple(want[big["id"]])
