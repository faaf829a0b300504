"""Served form on the GPU: jobs admitted by free bytes and stepped together are each bit-exact vs the oracle,
and a job's result is the same alone as in the mix."""
import pytest

import oracle as O
from paper_1809_07444_gb300 import workloads as WL
from paper_1809_07444_gb300.serve import WATOR, Server, summarize

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
    srv = Server(arena_bytes=6 << 20, gol_fraction=0.4, max_jobs=64)
    rep = srv.run(jobs, realtime=False)
    assert rep["unfinished"] == 0 and len(rep["done"]) == len(jobs)
    waited = [d for d in rep["done"] if d["admitted"] > 0.0 and d["admitted"] > min(x["completed"] for x in rep["done"])]
    assert waited, "expected some jobs to be admitted only after others completed"
    for d in rep["done"]:
        assert tuple(d["hash"]) == _oracle_hash(d), "job %d (app %d side %d)" % (d["id"], d["app"], d["side"])
    s = summarize(rep)
    assert s["jobs_done"] == 30 and s["step_ms_p99"] >= s["step_ms_p50"] > 0


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
