"""ctypes declarations of libdsr.so (include/dsr.h, include/dsr_apps.h).

Argument marshalling only. Loading fails loudly when the library has not
been built: there is no fallback.
"""
import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# DSR_LIBRARY=check selects the build with device self-checks (libdsr_check.so)
LIB_PATH = os.path.join(_PKG, "libdsr_check.so" if os.environ.get("DSR_LIBRARY") == "check" else "libdsr.so")

MAX_TYPES = 8
MAX_FIELDS = 16
MAX_LEVELS = 6

OK, E_INVALID, E_OOM, E_CUDA, E_DEVICE, E_TOO_LARGE = 0, 1, 2, 3, 4, 5
NOALLOC_MAX_SLOTS = 16384
CTR_COUNT = 8  # event counters per heap (DSR_CTR_COUNT)
ERR_OOM, ERR_RETRY, ERR_DOUBLE_FREE, ERR_BAD_HANDLE, ERR_CAPACITY = 1, 2, 4, 8, 16

METHOD_COUNT, METHOD_STREAM_ADD, METHOD_DELETE_IF, METHOD_CLONE = 1, 2, 3, 4
METHOD_GOL_COUNT, METHOD_GOL_DIE, METHOD_GOL_BIRTH = 100, 101, 102
METHOD_WATOR_F1, METHOD_WATOR_F2, METHOD_WATOR_S0, METHOD_WATOR_S1, METHOD_WATOR_S2 = 200, 201, 202, 203, 204
NULL_REF = 0xFFFFFFFFFFFFFFFF


class TypeDesc(C.Structure):
    _fields_ = [("name", C.c_char_p), ("n_fields", C.c_int), ("field_bytes", C.POINTER(C.c_int))]


class Tuning(C.Structure):
    _fields_ = [("cap_min", C.c_int), ("threads", C.c_int), ("ctas_per_sm", C.c_int), ("fanout", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n_blocks", C.c_uint64), ("free_blocks", C.c_uint64), ("n_types", C.c_uint32),
                ("error_flags", C.c_uint32), ("capacity", C.c_uint32 * MAX_TYPES),
                ("live_objects", C.c_uint64 * MAX_TYPES), ("allocated_blocks", C.c_uint64 * MAX_TYPES),
                ("active_blocks", C.c_uint64 * MAX_TYPES)]


class Layout(C.Structure):
    _fields_ = [("n_blocks", C.c_uint64), ("block_bytes", C.c_uint32), ("n_levels", C.c_uint32),
                ("words_per_level", C.c_uint64 * MAX_LEVELS), ("bitmap_words", C.c_uint64),
                ("off_free_bm", C.c_uint64), ("off_alloc_bm", C.c_uint64), ("off_active_bm", C.c_uint64),
                ("off_obj", C.c_uint64), ("off_type", C.c_uint64), ("off_data", C.c_uint64),
                ("arena_bytes_used", C.c_uint64), ("n_types", C.c_uint32),
                ("capacity", C.c_uint32 * MAX_TYPES), ("n_fields", C.c_uint32 * MAX_TYPES),
                ("field_bytes", (C.c_uint32 * MAX_FIELDS) * MAX_TYPES),
                ("field_offset", (C.c_uint32 * MAX_FIELDS) * MAX_TYPES), ("fanout", C.c_uint32),
                ("pad_", C.c_uint32)]


class WatorParams(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("seed", C.c_uint64), ("fish_breed", C.c_int32),
                ("shark_breed", C.c_int32), ("shark_energy0", C.c_int32), ("shark_gain", C.c_int32)]


class TrafficParams(C.Structure):
    _fields_ = [("R", C.c_int32), ("L", C.c_int32), ("vmax", C.c_int32), ("v_entry", C.c_int32),
                ("periodic", C.c_int32), ("pad_", C.c_int32), ("seed", C.c_uint64), ("p_thr", C.c_uint64),
                ("a_thr", C.c_uint64)]


class SugarscapeParams(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("seed", C.c_uint64), ("alpha", C.c_int32),
                ("endow_lo", C.c_int32), ("endow_hi", C.c_int32), ("metab_lo", C.c_int32), ("metab_hi", C.c_int32),
                ("vision_lo", C.c_int32), ("vision_hi", C.c_int32), ("age_lo", C.c_int32), ("age_hi", C.c_int32)]


NBODY_PAIRS_FP32, NBODY_PAIRS_FP64 = 0, 1


class NBodyParams(C.Structure):
    _fields_ = [("G", C.c_double), ("eps", C.c_double), ("dt", C.c_double), ("r_merge", C.c_double),
                ("r_near", C.c_double), ("pair_precision", C.c_int32), ("pad_", C.c_int32)]


class CountArgs(C.Structure):
    _fields_ = [("counter_dev", C.c_void_p)]


class DeleteIfArgs(C.Structure):
    _fields_ = [("modulus", C.c_int32), ("residue", C.c_int32)]


class CloneArgs(C.Structure):
    _fields_ = [("dst_type", C.c_int32), ("add", C.c_int32)]


class GolArgs(C.Structure):
    _fields_ = [("cell_ref_dev", C.c_void_p), ("W", C.c_int32), ("H", C.c_int32)]


# name -> (restype, argtypes)
_vp, _sz, _u64, _u32, _i = C.c_void_p, C.c_size_t, C.c_uint64, C.c_uint32, C.c_int
SIGNATURES = {
    "dsr_heap_bytes_for_blocks": (_i, [C.POINTER(TypeDesc), _i, _u64, C.POINTER(Tuning), C.POINTER(_sz)]),
    "dsr_heap_plan": (_i, [C.POINTER(TypeDesc), _i, _u64, C.POINTER(Tuning), C.POINTER(Layout)]),
    "dsr_heap_create": (_i, [C.POINTER(TypeDesc), _i, _vp, _sz, C.POINTER(Tuning), _vp, C.POINTER(_vp)]),
    "dsr_heap_destroy": (_i, [_vp]),
    "dsr_heap_reset": (_i, [_vp, _vp]),
    "dsr_heap_layout": (_i, [_vp, C.POINTER(Layout)]),
    "dsr_type_tree": (_i, [C.POINTER(TypeDesc), _i, C.POINTER(_i), C.POINTER(_u32)]),
    "dsr_heap_set_bases": (_i, [_vp, C.POINTER(_i)]),
    "dsr_dev_heap_size": (_sz, []),
    "dsr_heap_device_view": (_i, [_vp, _vp, _sz]),
    "dsr_heap_stats": (_i, [_vp, _vp, C.POINTER(Stats)]),
    "dsr_parallel_do": (_i, [_vp, _i, _i, _vp, _sz, _vp]),
    "dsr_doall_scan": (_i, [_vp, _i, _vp]),
    "dsr_doall_run": (_i, [_vp, _i, _i, _vp, _sz, _vp]),
    "dsr_heap_dump": (_i, [_vp, _i, _vp, _u64, _vp, _vp]),
    "dsr_row_words": (_i, [_vp, _i]),
    "dsr_heap_hash": (_i, [_vp, _i, _vp, _vp]),
    "dsr_heap_inject_oom": (_i, [_vp, _u32, _vp]),
    "dsr_heap_counters": (_i, [_vp, _vp, C.POINTER(_u64)]),
    "dsr_status_string": (C.c_char_p, [_i]),
    "dsr_last_cuda_error": (C.c_char_p, []),
    "dsr_bench_alloc": (_i, [_vp, _u64, _i, _u64, _vp, _vp]),
    "dsr_bench_free": (_i, [_vp, _u64, _vp, _vp]),
    "dsr_bench_churn": (_i, [_vp, _u64, _i, _u64, _vp, _vp, _vp]),
    "dsr_bench_fma": (_i, [_vp, _i, _i, _vp]),
    "dsr_bench_atomics": (_i, [_vp, _u64, _i, _i, _vp]),
    "dsr_gol_types": (_i, [C.POINTER(TypeDesc)]),
    "dsr_gol_workspace_bytes": (_i, [_i, _i, C.POINTER(_sz)]),
    "dsr_gol_create": (_i, [_vp, _i, _i, _vp, _vp, _vp, C.POINTER(_vp)]),
    "dsr_gol_step": (_i, [_vp, _i, _vp]),
    "dsr_gol_destroy": (_i, [_vp]),
    "dsr_wator_types": (_i, [C.POINTER(TypeDesc)]),
    "dsr_wator_workspace_bytes": (_i, [_vp, _i, _i, C.POINTER(_sz)]),
    "dsr_wator_create": (_i, [_vp, C.POINTER(WatorParams), _vp, _vp, _vp, C.POINTER(_vp)]),
    "dsr_wator_step": (_i, [_vp, _i, _vp]),
    "dsr_wator_kinds": (_i, [_vp, _vp, _vp]),
    "dsr_wator_destroy": (_i, [_vp]),
    "dsr_wator_phase_timing": (_i, [_vp, _i]),
    "dsr_wator_phase_select": (_i, [_vp, _i]),
    "dsr_wator_attach": (_i, [_vp, _vp, _vp, C.POINTER(_vp)]),
    "dsr_bm_heap_bytes": (_i, [C.POINTER(TypeDesc), _i, C.POINTER(_u64), C.POINTER(_sz)]),
    "dsr_bm_heap_create": (_i, [C.POINTER(TypeDesc), _i, C.POINTER(_u64), _vp, _sz, _vp, C.POINTER(_vp)]),
    "dsr_bm_heap_destroy": (_i, [_vp]),
    "dsr_bm_heap_stats": (_i, [_vp, _vp, C.POINTER(_u64), C.POINTER(_u32)]),
    "dsr_bm_heap_hash": (_i, [_vp, _i, _vp, _vp]),
    "dsr_bm_heap_counters": (_i, [_vp, _vp, C.POINTER(_u64)]),
    "dsr_wator_bm_workspace_bytes": (_i, [_vp, _i, _i, C.POINTER(_sz)]),
    "dsr_wator_bm_create": (_i, [_vp, _vp, _vp, _vp, _vp, C.POINTER(_vp)]),
    "dsr_wator_bm_step": (_i, [_vp, _i, _vp]),
    "dsr_wator_bm_destroy": (_i, [_vp]),
    "dsr_wator_static_bytes": (_i, [_i, _i, _i, C.POINTER(_sz)]),
    "dsr_wator_static_create": (_i, [_vp, _vp, _vp, _i, _vp, C.POINTER(_vp)]),
    "dsr_wator_static_step": (_i, [_vp, _i, _vp]),
    "dsr_wator_static_hash": (_i, [_vp, _vp, _vp]),
    "dsr_wator_static_state": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "dsr_wator_static_visits": (_i, [_vp, C.POINTER(_u64)]),
    "dsr_wator_static_destroy": (_i, [_vp]),
    "dsr_wator_phase_times": (_i, [_vp, C.POINTER(C.c_double), C.POINTER(_i)]),
    "dsr_nbody_types": (_i, [C.POINTER(TypeDesc)]),
    "dsr_nbody_workspace_bytes": (_i, [_vp, _u64, C.POINTER(_sz)]),
    "dsr_nbody_create": (_i, [_vp, C.POINTER(NBodyParams), _vp, _i, _vp, _u64, _vp, C.POINTER(_vp)]),
    "dsr_nbody_step": (_i, [_vp, _i, _vp]),
    "dsr_nbody_merge_log": (_i, [_vp, C.POINTER(_vp), C.POINTER(_vp)]),
    "dsr_nbody_near_pairs": (_i, [_vp, C.POINTER(_vp)]),
    "dsr_nbody_destroy": (_i, [_vp]),
    "dsr_nbody_step_noalloc": (_i, [_vp, C.POINTER(NBodyParams), _i, _u64, _vp, _u64, _vp, _vp]),
    "dsr_traffic_types": (_i, [C.POINTER(TypeDesc)]),
    "dsr_traffic_workspace_bytes": (_i, [C.POINTER(TrafficParams), C.POINTER(_sz)]),
    "dsr_traffic_create": (_i, [_vp, C.POINTER(TrafficParams), _vp, _vp, _vp, C.POINTER(_vp)]),
    "dsr_traffic_step": (_i, [_vp, _i, _vp]),
    "dsr_traffic_occupancy": (_i, [_vp, C.POINTER(_vp)]),
    "dsr_traffic_destroy": (_i, [_vp]),
    "dsr_sugarscape_types": (_i, [C.POINTER(TypeDesc)]),
    "dsr_sugarscape_workspace_bytes": (_i, [_vp, C.POINTER(SugarscapeParams), C.POINTER(_sz)]),
    "dsr_sugarscape_create": (_i, [_vp, C.POINTER(SugarscapeParams), _vp, _vp, C.c_int64, _vp, _vp,
                                   C.POINTER(_vp)]),
    "dsr_sugarscape_step": (_i, [_vp, _i, _vp]),
    "dsr_sugarscape_events": (_i, [_vp, _vp, C.POINTER(_u64)]),
    "dsr_sugarscape_sugar": (_i, [_vp, _vp, _vp]),
    "dsr_sugarscape_destroy": (_i, [_vp]),
    "dsr_group_create": (_i, [C.POINTER(TypeDesc), _i, _vp, _sz, _i, C.POINTER(Tuning), _vp, C.POINTER(_vp)]),
    "dsr_group_create_shared": (_i, [C.POINTER(TypeDesc), _i, _vp, _i, C.POINTER(Tuning), _vp, C.POINTER(_vp)]),
    "dsr_group_destroy": (_i, [_vp]),
    "dsr_group_add_heap": (_i, [_vp, _u64, _sz, _vp, C.POINTER(_i), C.POINTER(_vp), C.POINTER(_vp)]),
    "dsr_group_remove_heap": (_i, [_vp, _i]),
    "dsr_group_heap_bytes": (_i, [_vp, _u64, _sz, C.POINTER(_sz)]),
    "dsr_group_free_bytes": (_i, [_vp, C.POINTER(_sz), C.POINTER(_sz)]),
    "dsr_group_heap_count": (_i, [_vp]),
    "dsr_group_parallel_do": (_i, [_vp, _i, _i, _vp, _sz, _vp]),
    "dsr_group_check_record": (_i, [_vp, C.POINTER(_u32), C.POINTER(_u64)]),
    "dsr_heap_check_record": (_i, [_vp, C.POINTER(_u32), C.POINTER(_u64)]),
    "dsr_wator_batch_create": (_i, [_vp, _sz, _i, C.POINTER(Tuning), _vp, C.POINTER(_vp)]),
    "dsr_wator_batch_create_shared": (_i, [_vp, _i, C.POINTER(Tuning), _vp, C.POINTER(_vp)]),
    "dsr_wator_batch_prepare": (_i, [_vp]),
    "dsr_wator_batch_instance_bytes": (_i, [_vp, _i, _i, _u64, C.POINTER(_sz)]),
    "dsr_wator_batch_add": (_i, [_vp, C.POINTER(WatorParams), _u64, _vp, _vp, C.POINTER(_i)]),
    "dsr_wator_batch_remove": (_i, [_vp, _i]),
    "dsr_wator_batch_step": (_i, [_vp, _i, _vp]),
    "dsr_wator_batch_heap": (_i, [_vp, _i, C.POINTER(_vp)]),
    "dsr_wator_batch_kinds": (_i, [_vp, _i, _vp, _vp]),
    "dsr_wator_batch_group": (_i, [_vp, C.POINTER(_vp)]),
    "dsr_wator_batch_destroy": (_i, [_vp]),
    "dsr_gol_batch_create": (_i, [_vp, _sz, _i, C.POINTER(Tuning), _vp, C.POINTER(_vp)]),
    "dsr_gol_batch_create_shared": (_i, [_vp, _i, C.POINTER(Tuning), _vp, C.POINTER(_vp)]),
    "dsr_gol_batch_prepare": (_i, [_vp]),
    "dsr_gol_batch_instance_bytes": (_i, [_vp, _i, _i, _u64, C.POINTER(_sz)]),
    "dsr_gol_batch_add": (_i, [_vp, _i, _i, _u64, _vp, _vp, C.POINTER(_i)]),
    "dsr_gol_batch_remove": (_i, [_vp, _i]),
    "dsr_gol_batch_step": (_i, [_vp, _i, _vp]),
    "dsr_gol_batch_heap": (_i, [_vp, _i, C.POINTER(_vp)]),
    "dsr_gol_batch_group": (_i, [_vp, C.POINTER(_vp)]),
    "dsr_gol_batch_destroy": (_i, [_vp]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libdsr.so and declare its entry points. Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libdsr.so is not built (%s); run __graft_entry__.build()" % path)
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class DsrError(RuntimeError):
    pass


def check(rc, what=""):
    if rc != OK:
        L = load()
        msg = L.dsr_status_string(rc).decode()
        if rc == E_CUDA:
            msg += ": " + L.dsr_last_cuda_error().decode()
        raise DsrError("%s failed: %s (%d)" % (what, msg, rc))
