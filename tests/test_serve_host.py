"""CPU checks of the serving scheduler (paper_1809_07444_gb300/serve.py)
with fake batches in place of the GPU ones: first-fit admission by free
bytes (later small jobs may pass a large waiting one), the per-tick
admission bound, retirement after exactly `steps` ticks, and the report."""
import pytest

torch = pytest.importorskip("torch")

from paper_1809_07444_gb300 import serve  # noqa: E402


class FakeEvent:
    def __init__(self, enable_timing=False):
        pass

    def record(self, stream=None):
        pass

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return 1.0


class FakeHeap:
    def __init__(self, visits):
        self.v = visits

    def counters(self):
        return {"visits": self.v}


class FakeStream:
    def synchronize(self):
        pass


class FakeBatch:
    """Capacity in cells: a job of side s needs s * s. Batches made with
    share=other draw on the other's capacity (one arena)."""

    def __init__(self, capacity, share=None):
        self.capacity = capacity
        self.inst = {}  # slot -> (side, ticks stepped)
        self.next = 0
        self.log = []
        self.peers = share.peers if share else []
        self.peers.append(self)
        self.prepared = 0

    def used(self):
        return sum(s * s for b in self.peers for s, _ in b.inst.values())

    def prepare(self):
        self.prepared += 1

    def add(self, W, H, start, seed=None):
        if self.used() + W * H > self.capacity:
            return None
        slot = self.next
        self.next += 1
        self.inst[slot] = (W, 0)
        self.log.append(("add", slot, W))
        return slot

    def step(self, n=1):
        for k, (s, t) in list(self.inst.items()):
            self.inst[k] = (s, t + n)

    def heap(self, slot):
        return FakeHeap(self.inst[slot][1])

    def hash(self, slot):
        s, t = self.inst[slot]
        return (s, t)

    def remove(self, slot):
        self.log.append(("remove", slot))
        del self.inst[slot]


def _server(capacity, shared=False):
    s = serve.Server.__new__(serve.Server)
    s.wb = FakeBatch(capacity)
    s.gb = FakeBatch(capacity, share=s.wb if shared else None)
    s.stream = FakeStream()
    return s


@pytest.fixture(autouse=True)
def fake_cuda(monkeypatch):
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)


def _job(i, side, steps, app=serve.WATOR, arrival=0.0):
    return {"id": i, "arrival": arrival, "app": app, "side": side, "steps": steps, "seed": 100 + i}


def test_every_job_runs_exactly_its_steps():
    s = _server(capacity=3 * 32 * 32)
    jobs = [_job(i, 16 + 8 * (i % 3), 3 + i % 5, app=serve.WATOR if i % 2 else serve.GOL) for i in range(12)]
    rep = s.run(jobs, realtime=False, workers=2)
    assert rep["unfinished"] == 0 and len(rep["done"]) == 12
    for d in rep["done"]:
        side, ticks = d["hash"]  # the fake hash: (side, steps taken while resident)
        assert side == d["side"] and ticks == d["steps"]
    assert not s.wb.inst and not s.gb.inst  # every slot returned
    assert rep["visits"] == sum(d["steps"] for d in rep["done"])


def test_first_fit_lets_small_jobs_pass_a_large_one():
    s = _server(capacity=64 * 64)
    jobs = [_job(0, 40, 10), _job(1, 50, 2), _job(2, 16, 2), _job(3, 16, 2)]
    rep = s.run(jobs, realtime=False, workers=1)
    assert rep["unfinished"] == 0
    adds = [w for op, *rest in s.wb.log if op == "add" for w in rest[1:]]
    # 40 is admitted; 50 does not fit beside it and waits; the 16s pass it
    assert adds[:3] == [40, 16, 16] and adds[3] == 50
    done = {d["id"]: d for d in rep["done"]}
    assert done[1]["admitted"] >= done[2]["admitted"]


def test_admission_per_tick_is_bounded():
    s = _server(capacity=10 ** 9)
    jobs = [_job(i, 8, 4) for i in range(9)]
    resident_per_tick = []
    real_step = s.wb.step

    def step(n=1):
        resident_per_tick.append(len(s.wb.inst))
        real_step(n)
    s.wb.step = step
    rep = s.run(jobs, realtime=False, max_admit_per_tick=2, workers=1)
    assert rep["unfinished"] == 0
    assert all(b - a <= 2 for a, b in zip([0] + resident_per_tick, resident_per_tick))


def test_summary_of_a_report():
    s = _server(capacity=10 ** 9)
    rep = s.run([_job(i, 8, 2) for i in range(4)], realtime=False, workers=1)
    out = serve.summarize(rep)
    assert out["jobs_done"] == 4 and out["jobs_unfinished"] == 0 and out["ticks"] == len(rep["step_ms"]) > 0
    assert out["step_ms_p50"] == 1.0


def test_one_pool_for_both_applications():
    # with one shared arena a stream of one application can use all of it,
    # and the other application's jobs wait for those bytes
    s = _server(capacity=4 * 32 * 32, shared=True)
    jobs = [_job(i, 32, 3, app=serve.GOL) for i in range(4)] + [_job(9, 32, 2, app=serve.WATOR)]
    rep = s.run(jobs, realtime=False, workers=1)
    assert rep["unfinished"] == 0
    done = {d["id"]: d for d in rep["done"]}
    assert all(done[i]["admitted"] <= done[9]["admitted"] for i in range(4))
    assert done[9]["admitted"] >= min(done[i]["completed"] for i in range(4))
    assert s.gb.prepared > 0 and s.wb.prepared > 0


def test_report_times_admissions_and_retirements():
    s = _server(capacity=10 ** 9)
    rep = s.run([_job(i, 8, 2 + i) for i in range(5)], realtime=False, workers=1)
    out = serve.summarize(rep)
    assert len(rep["admit_ms"]) >= 1 and len(rep["retire_ms"]) >= 1
    assert out["admit_ms_p99"] >= out["admit_ms_p50"] >= 0 and 1 <= out["resident_max"] <= 5
    assert len(rep["resident"]) == out["ticks"] == len(rep["resident_cells"])
    assert out["step_ms_per_mcell_p50"] > 0 and out["admit_ms_per_job_p50"] >= 0
