"""CPU checks of the C ABI: the library builds, loads and exports every declared entry point;
host-only layout planning follows the block geometry of Section 2."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1809_07444_gb300 import build_ext, _lib

    build_ext.build()
    return _lib.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(dsr_[a-z0-9_]+)\s*\(", text, re.M):
            if not m.group(0).lstrip().startswith(("typedef", "#")):
                names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) > 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_declarations():
    from paper_1809_07444_gb300 import _lib

    assert set(_lib.SIGNATURES) <= _declared()


def _plan(lib, types, n_blocks, cap_min=0, fanout=0):
    from paper_1809_07444_gb300 import _lib as L
    from paper_1809_07444_gb300.heap import _descs

    descs, _keep = _descs(types)
    lay = L.Layout()
    tun = L.Tuning(cap_min, 0, 0, fanout)
    rc = lib.dsr_heap_plan(descs, len(types), n_blocks, C.byref(tun), C.byref(lay))
    return rc, lay


def test_capacity_rule(lib):
    # smallest type (8 B) gets 64 slots and fixes the block size; a 12 B
    # type gets floor(64*8/12) = 42, a 32 B type 16, a 16 B type 32
    rc, lay = _plan(lib, [[4, 4, 4], [4, 4], [4] * 8, [8, 8]], 1000)
    assert rc == 0
    assert [lay.capacity[t] for t in range(4)] == [42, 64, 16, 32]
    assert lay.block_bytes == 512
    # every SOA array starts 8-byte aligned and fits the block
    for t in range(4):
        offs = [lay.field_offset[t][f] for f in range(lay.n_fields[t])]
        assert all(o % 8 == 0 for o in offs)
        last = offs[-1] + lay.capacity[t] * lay.field_bytes[t][lay.n_fields[t] - 1]
        assert last <= lay.block_bytes


def test_cap_min_32_halves_blocks(lib):
    rc, lay = _plan(lib, [[4, 4, 4], [4, 4, 4, 4]], 1000, cap_min=32)
    assert rc == 0
    assert [lay.capacity[0], lay.capacity[1]] == [32, 24]
    assert lay.block_bytes == 384


def test_levels_and_offsets(lib):
    for M, levels in [(64, 1), (65, 2), (4096, 2), (4097, 3), (64 ** 3 + 1, 4)]:
        rc, lay = _plan(lib, [[4, 4]], M)
        assert rc == 0 and lay.n_levels == levels
        n, words = M, []
        while True:
            words.append(-(-n // 64))
            if n <= 64:
                break
            n = -(-n // 64)
        assert [lay.words_per_level[l] for l in range(levels)] == words
        assert lay.off_data % 1024 == 0 and lay.off_obj % 256 == 0
        assert lay.arena_bytes_used >= lay.off_data + M * lay.block_bytes


def test_invalid_descriptors_rejected(lib):
    assert _plan(lib, [[4, 3]], 10)[0] == 1
    assert _plan(lib, [[4] * 17], 10)[0] == 1
    assert _plan(lib, [[4]] * 9, 10)[0] == 1
    assert _plan(lib, [[4]], 0)[0] == 1
    assert _plan(lib, [[4]], 10, cap_min=48)[0] == 1


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_1809_07444_gb300 import _lib

    with pytest.raises(RuntimeError):
        _lib._lib = None
        try:
            _lib.load(str(tmp_path / "missing.so"))
        finally:
            _lib._lib = None


@pytest.mark.parametrize("fanout,words", [(0, [79, 2, 1]), (64, [79, 2, 1]), (32, [157, 5, 1]),
                                          (16, [313, 20, 2, 1])])
def test_bitmap_fanout_sets_the_level_structure(lib, fanout, words):
    rc, lay = _plan(lib, [[4, 4]], 5000, fanout=fanout)
    assert rc == 0
    assert lay.fanout == (fanout or 64)
    assert [lay.words_per_level[l] for l in range(lay.n_levels)] == words
    assert lay.bitmap_words == sum(words)


def test_bitmap_fanout_rejects_bad_widths_and_too_many_levels(lib):
    from paper_1809_07444_gb300 import _lib as L
    assert _plan(lib, [[4, 4]], 5000, fanout=8)[0] == L.E_INVALID
    # 16-bit containers reach DSR_MAX_LEVELS (6) levels at 16^6 blocks
    assert _plan(lib, [[4, 4]], 16 ** 6, fanout=16)[0] == 0
    assert _plan(lib, [[4, 4]], 16 ** 6 + 1, fanout=16)[0] == L.E_INVALID


def test_traffic_parameters_are_checked_on_the_host(lib):
    from paper_1809_07444_gb300 import _lib as L
    ok = L.TrafficParams(16, 100, 5, 5, 0, 0, 1, 1 << 30, 1 << 31)
    n = C.c_size_t(0)
    assert lib.dsr_traffic_workspace_bytes(C.byref(ok), C.byref(n)) == 0
    assert n.value == 2 * ((16 * 100 + 255) // 256 * 256)
    bad = [
        L.TrafficParams(16, 5, 5, 5, 0, 0, 1, 0, 0),           # road no longer than vmax
        L.TrafficParams(16, 100, 0, 0, 0, 0, 1, 0, 0),         # vmax 0
        L.TrafficParams(16, 100, 5, 6, 0, 0, 1, 0, 0),         # entry faster than vmax
        L.TrafficParams(0, 100, 5, 5, 0, 0, 1, 0, 0),          # no road
        L.TrafficParams(16, 100, 5, 5, 0, 0, 1, (1 << 32) + 1, 0),  # probability above 1
    ]
    for p in bad:
        assert lib.dsr_traffic_workspace_bytes(C.byref(p), C.byref(n)) == L.E_INVALID


def test_a_user_method_compiles_against_the_public_headers(tmp_path):
    # include/dsr_device.cuh is the interface for methods written outside the
    # library: a method struct, dsr_new / dsr_field, and the do-all kernel
    from paper_1809_07444_gb300 import build_ext
    import subprocess
    src = os.path.join(ROOT, "tests", "user_method.cu")
    r = subprocess.run([build_ext.nvcc(), "-c", src, "-o", str(tmp_path / "user_method.o"), "-std=c++17",
                        "-I", os.path.join(ROOT, "include"), "-Werror", "all-warnings"] + build_ext.ARCH,
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
