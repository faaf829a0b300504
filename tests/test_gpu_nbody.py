"""GPU (FP32) n-body with merging against the FP64 oracle: identical merges, state within 1e-4 relative."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1809_07444_gb300 import workloads as WL
from paper_1809_07444_gb300.apps import NBody

from helpers import check_invariants

pytestmark = pytest.mark.gpu

REL = 1e-4     # relative tolerance on position and velocity (FP32 vs FP64)
V_FLOOR = 1e-7  # absolute floor for velocities whose FP64 value is zero


def _compare(gpu_rows, ref_rows):
    assert np.array_equal(gpu_rows[:, 0], ref_rows[:, 0]), "live ids differ"
    assert np.array_equal(gpu_rows[:, 7].astype(np.float32), gpu_rows[:, 7])
    for cols in ((1, 4), (4, 7)):
        g, r = gpu_rows[:, cols[0]:cols[1]], ref_rows[:, cols[0]:cols[1]]
        err = np.linalg.norm(g - r, axis=1)
        scale = np.maximum(np.linalg.norm(r, axis=1), V_FLOOR)
        worst = (err / scale).max() if len(err) else 0.0
        assert worst <= REL, "relative error %.3g in columns %s" % (worst, cols)
    assert np.allclose(gpu_rows[:, 7], ref_rows[:, 7], rtol=REL, atol=0)


def _run(rows, steps, threads=8, **kw):
    O.set_threads(threads)
    gpu = NBody(rows, **kw)
    ref = O.NBody(rows, **kw)
    all_ref_merges = []
    for t in range(steps):
        gpu.step(1)
        mg, marg = ref.step(1, margin=1e-6)
        all_ref_merges.extend(mg.tolist())
        _compare(gpu.dump(), ref.dump())
    gm = gpu.merges()
    rm = np.array(sorted(map(tuple, all_ref_merges)), dtype=np.int64).reshape(-1, 3)
    assert np.array_equal(gm, rm), "merge logs differ"
    st = gpu.heap.stats()
    assert st["error_flags"] == 0
    check_invariants(gpu.heap, [ref.count()])
    return gpu, ref, rm


def test_two_body_and_chain_cases():
    rows = np.zeros((3, 7))
    rows[:, 0] = [0.5, 0.5015, 0.503]
    rows[:, 1:3] = 0.5
    rows[:, 6] = [1.0, 3.0, 1.0]
    rows = rows.astype(np.float32).astype(np.float64)
    _, _, m = _run(rows, 2, G=0.0, r_merge=2e-3)
    assert m.tolist() == [[0, 0, 1], [1, 0, 2]]


def test_small_cluster_many_merges():
    # a dense cluster (1500 bodies in a box 0.06 wide) with a larger merge
    # distance: many merges in the first steps. Later steps of such a cluster
    # are chaotic close encounters where FP32 cannot follow FP64 to 1e-4, so
    # the comparison stops after the first step.
    rng = np.random.default_rng(0)
    n = 1500
    rows = np.zeros((n, 7))
    rows[:, 0:3] = 0.5 + 0.06 * rng.random((n, 3))
    rows[:, 6] = 10 ** rng.uniform(-3, 0, n)
    rows = rows.astype(np.float32).astype(np.float64)
    gpu, ref, m = _run(rows, 1, r_merge=3e-3)
    assert len(m) > 10


@pytest.mark.parametrize("n,seed", [(1, 1), (63, 2), (4097, 3)])
def test_ragged_counts_against_oracle(n, seed):
    rows, _ = WL.nbody_initial(n, seed)
    _run(rows, 5)


def test_full_size_65536_bodies_first_steps():
    # the 65,536-body workload: positions uniform in the unit cube, masses
    # log-uniform in [1e-3, 1], G = 1, eps = 1e-3, dt = 1e-4, merge distance
    # 2e-3; identical merges and state within 1e-4 for the first 3 steps
    rows, _ = WL.nbody_initial(65536, 1)
    _, _, m = _run(rows, 3, threads=os.cpu_count() or 8)
    assert len(m) > 100


@pytest.mark.xfail(strict=True, reason=(
    "FP32 state cannot follow the FP64 trajectory through close encounters for 50 steps: "
    "measured on GB300, first body beyond 1e-4 relative velocity error at step 4 (5 of 64,762 bodies), "
    "first differing merge decision at step 7"))
def test_full_size_65536_bodies_50_steps():
    # the full 50-step comparison, kept at the 1e-4 bar; expected to fail
    rows, _ = WL.nbody_initial(65536, 1)
    _run(rows, 50, threads=os.cpu_count() or 8)
