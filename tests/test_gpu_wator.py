"""GPU parity of wa-tor with the oracle (bit-exact Fish and Shark multisets, state hash every step)."""
import numpy as np
import pytest

import oracle as O
from paper_1809_07444_gb300 import _lib as L
from paper_1809_07444_gb300 import workloads as WL
from paper_1809_07444_gb300.apps import Wator

from helpers import check_invariants

pytestmark = pytest.mark.gpu


def _run_pair(W, H, kind0, seed, steps, full_every=1, invariants_every=None):
    gpu, ref = Wator(W, H, kind0, seed), O.Wator(W, H, kind0, seed)
    assert gpu.hash() == ref.hash()
    for t in range(1, steps + 1):
        c0 = gpu.heap.counters()
        gpu.step(1)
        ev = ref.step(1)[0]
        c1 = gpu.heap.counters()
        # event counters: moves, births and deaths of the step
        assert c1["app0"] - c0["app0"] == ev[4] + ev[5], "moves at step %d" % t
        assert c1["allocs"] - c0["allocs"] == ev[0] + ev[2], "births at step %d" % t
        assert c1["frees"] - c0["frees"] == ev[1] + ev[3], "deaths at step %d" % t
        hg, hr = gpu.hash(), ref.hash()
        assert hg == hr, "step %d: hash %s vs oracle %s" % (t, hg, hr)
        if t % full_every == 0 or t == steps:
            fg, sg = gpu.dump()
            fr, sr = ref.dump()
            assert np.array_equal(fg, fr), "fish differ at step %d" % t
            assert np.array_equal(sg, sr), "sharks differ at step %d" % t
            assert np.array_equal(gpu.grid(), ref.grid())
        if invariants_every and t % invariants_every == 0:
            check_invariants(gpu.heap, list(ref.counts()))
    st = gpu.heap.stats()
    assert st["error_flags"] == 0, st
    check_invariants(gpu.heap, list(ref.counts()))
    return gpu, ref


def test_wator_64x64_bit_exact():
    _run_pair(64, 64, WL.wator_initial(64, 64, 1), 1, 150, full_every=10, invariants_every=25)


@pytest.mark.parametrize("W,H,seed,steps", [(3, 3, 2, 30), (17, 9, 3, 80), (257, 129, 4, 60)])
def test_wator_ragged_grids(W, H, seed, steps):
    _run_pair(W, H, WL.wator_initial(W, H, seed), seed, steps, full_every=10)


def test_wator_extinction_and_degenerate_starts():
    # no agents; only sharks (they all starve); only fish (fill the grid)
    _run_pair(32, 32, np.zeros((32, 32), np.uint8), 1, 5)
    k = np.zeros((32, 32), np.uint8)
    k[::3, ::2] = 2
    gpu, ref = _run_pair(32, 32, k, 2, 8)
    assert ref.counts() == (0, 0)
    k = np.zeros((32, 32), np.uint8)
    k[5, 5] = 1
    _run_pair(32, 32, k, 3, 40, full_every=5)


def test_wator_phase_timing_records_every_step():
    w = Wator(64, 64, WL.wator_initial(64, 64, 1), 1)
    w.phase_timing(4)
    w.step(6)  # events for the first four only
    run, scan, n = w.phase_times()
    assert n == 4 and all(v > 0 for v in run.values()) and all(v > 0 for v in scan.values())
    w.step(2)
    assert w.phase_times()[2] == 2  # a new window reuses the events
    w.phase_timing(0)
    w.step(1)
    assert w.phase_times()[2] == 0


def test_wator_phase_select_times_one_method_kernel():
    w = Wator(64, 64, WL.wator_initial(64, 64, 1), 1)
    w.phase_timing(6)
    w.step(2)
    w.phase_select(1)  # F2 only; drops the two steps above
    w.step(3)
    run, scan, n = w.phase_times()
    assert n == 3 and run["F2"] > 0
    assert all(v == 0 for p, v in run.items() if p != "F2") and all(v == 0 for v in scan.values())
    w.phase_select(None)
    w.step(1)
    run, scan, n = w.phase_times()
    assert n == 1 and all(v > 0 for v in run.values())
    with pytest.raises(L.DsrError):
        w.phase_select(5)


def test_wator_steps_inside_a_caller_graph_capture_match():
    # dsr_wator_step replays its own captured graph, except while the
    # caller's stream is being captured: then its kernels go into the
    # caller's graph, whose replays must advance the simulation exactly as
    # stepping does
    import ctypes as C

    import torch
    from paper_1809_07444_gb300.heap import _stream_ptr
    lib = L.load()
    k0 = WL.wator_initial(128, 128, 3)
    a = Wator(128, 128, k0, 3)
    b = Wator(128, 128, k0, 3)
    torch.cuda.synchronize()  # both initialised on the default stream
    s = torch.cuda.Stream()
    a.step(2)
    with torch.cuda.stream(s):
        L.check(lib.dsr_wator_step(b.handle, 2, _stream_ptr(s)), "dsr_wator_step")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        L.check(lib.dsr_wator_step(b.handle, 1, _stream_ptr(s)), "dsr_wator_step")
    for _ in range(6):
        a.step(1)
        with torch.cuda.stream(s):
            g.replay()
        torch.cuda.synchronize()
        assert a.hash() == b.hash()
    fa, sa = a.dump()
    fb, sb = b.dump()
    assert np.array_equal(fa, fb) and np.array_equal(sa, sb)
    assert a.heap.stats()["error_flags"] == 0 and b.heap.stats()["error_flags"] == 0
    del g


def test_wator_2048_full_size_all_500_steps():
    # the 2048 x 2048 workload (30% fish, 3% sharks) for its full 500 steps:
    # state hash and event counts every step, full multisets and the grid
    # every 50 steps, heap invariants every 100
    W = H = 2048
    _run_pair(W, H, WL.wator_initial(W, H, 1), 1, 500, full_every=50, invariants_every=100)


def test_wator_checkpoint_and_resume_bit_exact():
    W, H = 200, 150
    k0 = WL.wator_initial(W, H, 8)
    a, ref = Wator(W, H, k0, 8, tuning={"fanout": 32}), O.Wator(W, H, k0, seed=8)
    a.step(25)
    ref.step(25)
    ck = a.checkpoint()
    a.step(25)
    b = Wator.restore(ck)
    b.step(25)
    ref.step(25)
    assert a.hash() == b.hash() == ref.hash()
    fa, sa = a.dump()
    fb, sb = b.dump()
    assert np.array_equal(fa, fb) and np.array_equal(sa, sb)
    check_invariants(b.heap, list(ref.counts()))
