"""A do-all method written outside the library runs on the GPU (Section 2.3:
run a method in parallel for all objects of a type; Section 1.2: new inside
methods).

tests/user_method.cu uses only the public headers: it takes the heap's
device view (dsr_heap_device_view), lists the live blocks with the library's
scan (dsr_doall_scan), and launches dsr_doall_kernel over its own method,
which scales field 0 and creates a new object wherever the result passes
100. The test links it against libdsr.so, runs it on a heap whose field
values it wrote itself, and checks every object against the host's
expectation: each listed object scaled once, one new object (value 1) per
value above 100, none of the new ones visited, the block list reset for the
next do-all, and the heap's invariants and statistics intact.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest
import torch

from paper_1809_07444_gb300 import _lib as L
from paper_1809_07444_gb300 import build_ext
from paper_1809_07444_gb300.heap import Heap, _stream_ptr, heap_bytes_for_blocks

from helpers import check_invariants, check_stats

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def user_lib(tmp_path_factory):
    L.load()  # the user library binds to this already-loaded libdsr
    out = str(tmp_path_factory.mktemp("user") / "libuser_method.so")
    libdir, libname = os.path.split(L.LIB_PATH)
    cmd = [build_ext.nvcc(), "-shared", "-Xcompiler", "-fPIC", "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "user_method.cu"), "-o", out, "-L", libdir, "-l:" + libname,
           "-Xlinker", "-rpath=" + libdir, "-cudart", "shared"] + build_ext.ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    lib = C.CDLL(out)
    lib.user_scale.restype = C.c_int
    lib.user_scale.argtypes = [C.c_void_p, C.c_int, C.c_float, C.c_int, C.c_void_p]
    return lib


def _field0_offsets(heap, refs):
    """Byte offsets in the arena of field 0 of the objects `refs` (type 0)."""
    lay = heap.layout()
    r = refs.astype(np.uint64)
    return (int(lay.off_data) + (r >> np.uint64(6)).astype(np.int64) * int(lay.block_bytes)
            + int(lay.field_offset[0][0]) + (r & np.uint64(63)).astype(np.int64) * 4)


def _values(heap):
    f, _ = heap.dump(0)
    return np.sort(f[:, 0].view(np.float32))


def test_user_method_scales_each_object_once_and_news_are_not_visited(user_lib):
    types = [[4], [4, 4]]
    heap = Heap(types, heap_bytes_for_blocks(types, 8000))
    n = 200_000
    refs_t = torch.empty(n, dtype=torch.int64, device="cuda")
    heap.bench_alloc(refs_t, 1, 5)
    refs = refs_t.cpu().numpy().view(np.uint64)
    assert len(np.unique(refs)) == n
    # write known values into field 0 of every object
    rng = np.random.default_rng(7)
    v0 = (rng.random(n) * 60.0).astype(np.float32)
    off = _field0_offsets(heap, refs)
    heap.arena.view(torch.float32)[torch.from_numpy(off // 4).cuda()] = torch.from_numpy(v0).cuda()
    torch.cuda.synchronize()
    sm = torch.cuda.get_device_properties(0).multi_processor_count

    # first do-all: scale by 2.5; values above 100 create a new object
    rc = user_lib.user_scale(heap.handle.value, 0, 2.5, 4 * sm, _stream_ptr())
    assert rc == 0
    torch.cuda.synchronize()
    v1 = v0 * np.float32(2.5)
    n_new = int((v1 > np.float32(100.0)).sum())
    assert 0 < n_new < n
    got = heap.arena.view(torch.float32)[torch.from_numpy(off // 4).cuda()].cpu().numpy()
    assert np.array_equal(got, v1), "an object was not scaled exactly once"
    want = np.sort(np.concatenate([v1, np.ones(n_new, np.float32)]))  # the new ones were not visited
    assert np.array_equal(_values(heap), want)
    # the method kernel reset the block list: the library's next do-all sees
    # exactly the live set
    assert heap.count(0) == n + n_new
    st = check_stats(heap)
    assert st["live_objects"] == [n + n_new, 0] and st["error_flags"] == 0
    check_invariants(heap, [n + n_new, 0])

    # second do-all over everything, new objects included: halve, no births
    rc = user_lib.user_scale(heap.handle.value, 0, 0.5, 2 * sm, _stream_ptr())
    assert rc == 0
    torch.cuda.synchronize()
    assert np.array_equal(_values(heap), np.sort(want * np.float32(0.5)))
    assert heap.count(0) == n + n_new
    check_stats(heap)


def test_user_method_on_an_empty_type_is_a_no_op(user_lib):
    types = [[4], [4, 4]]
    heap = Heap(types, heap_bytes_for_blocks(types, 64))
    rc = user_lib.user_scale(heap.handle.value, 0, 3.0, 8, _stream_ptr())
    assert rc == 0
    torch.cuda.synchronize()
    assert heap.count(0) == 0
    check_stats(heap)
