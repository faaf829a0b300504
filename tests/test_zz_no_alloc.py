"""The allocation-free n-body step (dsr_nbody_step_noalloc).

Some callers cannot call cudaMalloc: a plugin that is handed its device
memory by a host program which owns all of it, for example. For them
dsr_nbody_step_noalloc keeps the step's scratch in a static device array of
the library instead of a caller-allocated workspace. This test drives it
through the C ABI, one step per call, for five calls in a row, and after
every call checks it against the workspace-based dsr_nbody_step on an
identical heap and against the FP64 oracle, within the n-body tolerance of
the other tests (1e-4 relative, identical merges). From the second call on
it also checks that a call leaves the device's free memory unchanged. It is
collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from paper_1809_07444_gb300 import _lib as L
from paper_1809_07444_gb300.apps import NBody
from paper_1809_07444_gb300.heap import _stream_ptr

pytestmark = pytest.mark.gpu

REL = 1e-4


def _rows(n, seed):
    # a 0.2-wide cube, so that pairs come within the merge distance and
    # within the near-field radius
    rng = np.random.default_rng(seed)
    rows = np.zeros((n, 7))
    rows[:, 0:3] = 0.4 + 0.2 * rng.random((n, 3))
    rows[:, 6] = 10 ** rng.uniform(-3, 0, n)
    return rows.astype(np.float32).astype(np.float64)


def _close(a, b):
    assert np.array_equal(a[:, 0], b[:, 0]), "live ids differ"
    for lo, hi in ((1, 4), (4, 7)):
        err = np.linalg.norm(a[:, lo:hi] - b[:, lo:hi], axis=1)
        scale = np.maximum(np.linalg.norm(b[:, lo:hi], axis=1), 1e-7)
        assert (err / scale).max() <= REL
    assert np.allclose(a[:, 7], b[:, 7], rtol=REL, atol=0)


def _sorted(log):
    return log[np.lexsort(log.T[::-1])] if len(log) else log


def test_noalloc_step_matches_workspace_step_and_oracle_on_five_calls():
    lib = L.load()
    rows = _rows(4000, 21)
    ref = NBody(rows)    # stepped by dsr_nbody_step with its workspace
    other = NBody(rows)  # same bodies; stepped by dsr_nbody_step_noalloc
    p = other.params
    orc = O.NBody(rows, G=p.G, eps=p.eps, dt=p.dt, r_merge=p.r_merge)
    assert other.heap.layout().n_blocks * 64 <= L.NOALLOC_MAX_SLOTS
    log_cap = 4096
    log = torch.zeros(log_cap * 3, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    sp = _stream_ptr()
    orc_merges = []
    free_after = []
    for call in range(5):
        ref.step(1)
        orc_merges.extend(orc.step(1)[0].tolist())
        rc = lib.dsr_nbody_step_noalloc(other.heap.handle, C.byref(p), 1, call, C.c_void_p(log.data_ptr()), log_cap,
                                        C.c_void_p(count.data_ptr()), sp)
        assert rc == L.OK, lib.dsr_status_string(rc)
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0])
        got = other.dump()
        _close(got, ref.dump())
        _close(got, orc.dump())
        n = int(count.item())
        mine = _sorted(log[: 3 * n].cpu().numpy().reshape(n, 3).astype(np.int64))
        assert np.array_equal(mine, ref.merges())
        assert np.array_equal(mine, np.array(sorted(map(tuple, orc_merges)), dtype=np.int64).reshape(-1, 3))
    assert len(orc_merges) > 0
    # the first call may load the library's kernels; later calls allocate nothing
    assert len(set(free_after[1:])) == 1, free_after
    assert other.heap.stats()["error_flags"] == 0


def test_noalloc_fp64_pair_forces_match_the_oracle():
    # the same entry point with FP64 pair forces, two calls of three steps
    lib = L.load()
    rows = _rows(3000, 5)
    other = NBody(rows, pairs="fp64")
    p = other.params
    orc = O.NBody(rows, G=p.G, eps=p.eps, dt=p.dt, r_merge=p.r_merge)
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    log = torch.zeros(4096 * 3, dtype=torch.int32, device="cuda")
    merges = []
    for call in range(2):
        rc = lib.dsr_nbody_step_noalloc(other.heap.handle, C.byref(p), 3, 3 * call, C.c_void_p(log.data_ptr()), 4096,
                                        C.c_void_p(count.data_ptr()), _stream_ptr())
        assert rc == L.OK, lib.dsr_status_string(rc)
        merges.extend(orc.step(3)[0].tolist())
        torch.cuda.synchronize()
        _close(other.dump(), orc.dump())
    n = int(count.item())
    mine = _sorted(log[: 3 * n].cpu().numpy().reshape(n, 3).astype(np.int64))
    assert np.array_equal(mine, np.array(sorted(map(tuple, merges)), dtype=np.int64).reshape(-1, 3))


def test_noalloc_rejects_heaps_beyond_its_maximum():
    lib = L.load()
    big = NBody(_rows(20000, 3))
    assert big.heap.layout().n_blocks * 64 > L.NOALLOC_MAX_SLOTS
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = lib.dsr_nbody_step_noalloc(big.heap.handle, C.byref(big.params), 1, 0, None, 0,
                                    C.c_void_p(count.data_ptr()), _stream_ptr())
    assert rc == L.E_TOO_LARGE
