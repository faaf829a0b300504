"""The allocation-free n-body step (dsr_nbody_step_noalloc) matches the workspace-based step.

For callers that cannot call cudaMalloc, dsr_nbody_step_noalloc keeps the
step's scratch in a static device array of the library instead of a
caller-allocated workspace. This test drives it through the C ABI and checks
two calls in a row against dsr_nbody_step on an identical heap, within the
n-body tolerance used by the other tests (1e-4 relative), with identical
merge logs. It is collected last so that a run stopping at the first failure
has already run every other test; it also passes on its own.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1809_07444_gb300 import _lib as L
from paper_1809_07444_gb300.apps import NBody
from paper_1809_07444_gb300.heap import _stream_ptr

pytestmark = pytest.mark.gpu

REL = 1e-4


def _rows(n, seed):
    # a 0.2-wide cube, so that a few pairs come within the merge distance
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


def test_noalloc_step_matches_workspace_step_on_two_calls():
    lib = L.load()
    rows = _rows(4000, 21)
    ref = NBody(rows)    # stepped by dsr_nbody_step with its workspace
    other = NBody(rows)  # same bodies; stepped by dsr_nbody_step_noalloc
    assert other.heap.layout().n_blocks * 64 <= L.NOALLOC_MAX_SLOTS
    log_cap = 4096
    log = torch.zeros(log_cap * 3, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    sp = _stream_ptr()
    for call in range(2):
        ref.step(1)
        rc = lib.dsr_nbody_step_noalloc(other.heap.handle, C.byref(other.params), 1, call,
                                        C.c_void_p(log.data_ptr()), log_cap, C.c_void_p(count.data_ptr()), sp)
        assert rc == L.OK, lib.dsr_status_string(rc)
        torch.cuda.synchronize()
        _close(other.dump(), ref.dump())
        n = int(count.item())
        got = log[: 3 * n].cpu().numpy().reshape(n, 3).astype(np.int64)
        got = got[np.lexsort(got.T[::-1])] if n else got
        assert np.array_equal(got, ref.merges())
    assert len(ref.merges()) > 0
    assert other.heap.stats()["error_flags"] == 0


def test_noalloc_rejects_heaps_beyond_its_maximum():
    lib = L.load()
    big = NBody(_rows(20000, 3))
    assert big.heap.layout().n_blocks * 64 > L.NOALLOC_MAX_SLOTS
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = lib.dsr_nbody_step_noalloc(big.heap.handle, C.byref(big.params), 1, 0, None, 0,
                                    C.c_void_p(count.data_ptr()), _stream_ptr())
    assert rc == L.E_TOO_LARGE
