"""Batched wa-tor on the GPU: every instance of a graph-captured group step matches its own oracle run.

The instances have their own heaps in one arena (a heap group); one batched
step is five group do-alls over all of them. Each instance must give exactly
the result it gives alone.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as O
from paper_1809_07444_gb300 import workloads as WL
from paper_1809_07444_gb300.apps import Wator, WatorBatch

from helpers import check_invariants

pytestmark = pytest.mark.gpu


def _oracle_hashes(args):
    """Run one oracle instance; hashes after each checkpoint step (runs in a spawned worker)."""
    side, seed, steps, checkpoints = args
    import oracle as Ow
    from paper_1809_07444_gb300 import workloads as WLw
    w = Ow.Wator(side, side, WLw.wator_initial(side, side, seed), seed=seed)
    out, done = [], 0
    for c in checkpoints:
        w.step(c - done)
        done = c
        out.append(w.hash())
    return out, w.counts()


def test_batch_matches_oracle_every_step():
    sides = [16, 23, 37, 64, 3, 100, 128, 5, 77, 41]
    b = WatorBatch(256 << 20, max_instances=16)
    refs, slots = [], []
    for i, s in enumerate(sides):
        k0 = WL.wator_initial(s, s, 100 + i)
        slots.append(b.add(s, s, k0, 100 + i))
        refs.append(O.Wator(s, s, k0, seed=100 + i))
    for t in range(1, 61):
        b.step(1)
        for slot, ref in zip(slots, refs):
            ref.step(1)
            assert b.hash(slot) == ref.hash(), "instance %d, step %d" % (slot, t)
    for slot, ref in zip(slots, refs):
        f, s = b.dump(slot)
        fr, sr = ref.dump()
        assert np.array_equal(f, fr) and np.array_equal(s, sr)
        assert np.array_equal(b.grid(slot), ref.grid())
        hp = b.heap(slot)
        assert hp.stats()["error_flags"] == 0
        check_invariants(hp, list(ref.counts()))


def test_instances_join_and_leave_between_steps():
    b = WatorBatch(128 << 20, max_instances=8)
    k = {s: WL.wator_initial(s, s, s) for s in (20, 30, 40)}
    a = b.add(20, 20, k[20], 20)
    ra = O.Wator(20, 20, k[20], seed=20)
    c = b.add(30, 30, k[30], 30)
    b.step(10)
    ra.step(10)
    b.remove(c)  # leaves; its bytes return to the arena
    d = b.add(40, 40, k[40], 40)  # joins later and starts at its own step 0
    rd = O.Wator(40, 40, k[40], seed=40)
    for _ in range(15):
        b.step(1)
        ra.step(1)
        rd.step(1)
        assert b.hash(a) == ra.hash() and b.hash(d) == rd.hash()
    b.remove(a)
    b.remove(d)
    total, largest = b.free_bytes()
    assert total == largest  # everything coalesced back into one range


def test_batch_equals_plain_form():
    side, seed = 96, 7
    k0 = WL.wator_initial(side, side, seed)
    b = WatorBatch(64 << 20, max_instances=4)
    slot = b.add(side, side, k0, seed)
    alone = Wator(side, side, k0, seed)
    for _ in range(40):
        b.step(1)
        alone.step(1)
        assert b.hash(slot) == alone.hash()


def test_arena_full_is_reported():
    b = WatorBatch(8 << 20, max_instances=64)
    added = 0
    while b.add(64, 64, WL.wator_initial(64, 64, added), added) is not None:
        added += 1
        assert added < 64
    assert added >= 1
    b.step(3)


def test_batched_256_instances_500_steps():
    # the batched workload: 256 instances, sides log-uniform in [64, 1024],
    # per-instance seeds; state hash of every instance at 5 checkpoints and at
    # step 500 against its own oracle run
    sides = WL.batched_sides(256, 1)
    seeds = [1000 + i for i in range(256)]
    checkpoints = [1, 10, 100, 250, 500]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(32, os.cpu_count() or 4)) as pool:
        pending = pool.map_async(_oracle_hashes, [(int(s), sd, 500, checkpoints) for s, sd in zip(sides, seeds)])
        need = sum(WatorBatch.blocks_for(int(s), int(s)) * 1000 + int(s) * int(s) * 24 for s in sides)
        b = WatorBatch(need + (256 << 20), max_instances=256)
        slots = [b.add(int(s), int(s), WL.wator_initial(int(s), int(s), sd), sd) for s, sd in zip(sides, seeds)]
        assert all(x is not None for x in slots)
        got, done = [], 0
        for c in checkpoints:
            b.step(c - done)
            done = c
            got.append([b.hash(x) for x in slots])
        want = pending.get()
    for i in range(256):
        for k in range(len(checkpoints)):
            assert got[k][i] == want[i][0][k], "instance %d (side %d) at step %d" % (i, sides[i], checkpoints[k])
        assert b.counts(slots[i]) == tuple(want[i][1])
    for x in slots[:8]:
        check_invariants(b.heap(x))
