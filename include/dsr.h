/*
 * dsr.h -- C ABI of the GB300 SOA object heap and parallel do-all.
 *
 * A from-scratch sm_103a implementation of the data-parallel hot path of
 * DynaSOAr (Springer, "DynaSOAr: Accelerating Single-Method Multiple-Objects
 * Applications on GPUs", arXiv 1809.07444):
 *   - a heap of equal-size blocks, each holding objects of one declared type
 *     in structure-of-arrays layout (Section 2, "The DynaSOAr System");
 *   - lock-free hierarchical bitmaps indexing the block states free,
 *     allocated[T] and active[T] (Section 2 "Block States", Section 3);
 *   - device-side new/delete (Alg. 1; declared in dsr_device.cuh);
 *   - the parallel do-all that runs a method on every object of a type
 *     (Section 2.3, Fig. 4).
 *
 * Conventions for every entry point
 *   - Pointers named *_dev or documented "device" are CUDA device pointers;
 *     everything else is host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Calls are asynchronous on that stream unless documented to
 *     synchronise. Calls on one heap must be ordered on one stream at a time.
 *   - The caller owns every device buffer it passes (the arena, workspaces,
 *     outputs) and must keep it alive until the work queued on the stream has
 *     finished. The library owns only the host-side handle it returns.
 *   - Return value: DSR_OK or one of the DSR_E_* codes below; nothing aborts.
 *     Errors found on the device (out of memory inside a kernel, a retry
 *     limit reached, a double free) are sticky bits in the heap, read back by
 *     dsr_heap_stats.
 */
#ifndef DSR_H
#define DSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DSR_MAX_TYPES 8
#define DSR_MAX_FIELDS 16
#define DSR_MAX_LEVELS 6

/* Status codes. */
enum {
    DSR_OK = 0,
    DSR_E_INVALID = 1,   /* bad argument: null pointer, bad type/method id, size out of range */
    DSR_E_OOM = 2,       /* arena too small for even one block per type */
    DSR_E_CUDA = 3,      /* a CUDA runtime call failed; see dsr_last_cuda_error */
    DSR_E_DEVICE = 4,    /* a device-side error bit is set (see dsr_stats.error_flags) */
    DSR_E_TOO_LARGE = 5  /* the problem exceeds a fixed maximum of the called entry point */
};

/* Event counters (dsr_heap_counters), cumulative since create or reset. */
#define DSR_CTR_VISITS 0u  /* objects visited by do-all method kernels */
#define DSR_CTR_ALLOCS 1u  /* objects created by dsr_new */
#define DSR_CTR_FREES 2u   /* objects deleted by dsr_delete */
#define DSR_CTR_BLOCKS 3u  /* blocks taken from the free bitmap (slow path) */
#define DSR_CTR_APP0 4u    /* 4 .. 7: counted by applications (wa-tor: successful moves) */
#define DSR_CTR_COUNT 8u

/* Device-side sticky error bits (dsr_stats.error_flags). */
#define DSR_ERR_OOM 1u          /* dsr_new found no free block; it returned DSR_NULL */
#define DSR_ERR_RETRY 2u        /* a bounded retry loop gave up (contention or inconsistency) */
#define DSR_ERR_DOUBLE_FREE 4u  /* dsr_delete of a slot that was already free */
#define DSR_ERR_BAD_HANDLE 8u   /* dsr_delete of a handle outside the heap */
#define DSR_ERR_CAPACITY 16u    /* an output buffer given to a dump was too small */

/* One declared object type (Section 2: all types are declared with the
 * allocator up front). Fields are 4 or 8 bytes; each becomes one SOA array
 * inside every block of this type. */
typedef struct {
    const char* name;        /* informational, may be NULL */
    int n_fields;            /* 1 .. DSR_MAX_FIELDS */
    const int* field_bytes;  /* n_fields entries, each 4 or 8 */
} dsr_type_desc;

/* Tuning knobs; pass NULL for the defaults. */
typedef struct {
    int cap_min;        /* slots per block of the smallest type: 64 (paper, default) or 32 */
    int threads;        /* threads per CTA of do-all kernels: 64..1024, multiple of 64 (default 256) */
    int ctas_per_sm;    /* persistent do-all grid = ctas_per_sm x SM count (0 = occupancy limit) */
    int fanout;         /* bits used per bitmap container (Section 2.1): 64 (paper, default), 32 or 16;
                           0 = default. Smaller containers mean more levels but fewer searchers per word. */
} dsr_tuning;

typedef struct dsr_heap dsr_heap;

/* Per-heap statistics (the space-efficiency view of Section 4). */
typedef struct {
    uint64_t n_blocks;                          /* M */
    uint64_t free_blocks;
    uint32_t n_types;
    uint32_t error_flags;                       /* DSR_ERR_* bits, sticky */
    uint32_t capacity[DSR_MAX_TYPES];           /* slots per block of each type */
    uint64_t live_objects[DSR_MAX_TYPES];
    uint64_t allocated_blocks[DSR_MAX_TYPES];
    uint64_t active_blocks[DSR_MAX_TYPES];
} dsr_stats;

/* Where each metadata array lives inside the arena (byte offsets from the
 * arena base), for inspection of a quiescent heap. Every bitmap has the same
 * level structure: level l has words_per_level[l] 64-bit words, of which the
 * low `fanout` bits are used (bit p of level l lives in word p / fanout, bit
 * p % fanout), levels are stored back to back (level 0 first), bitmap_words
 * in total. The
 * allocated[T] bitmaps are stored back to back in type order, as are the
 * active[T] bitmaps. */
typedef struct {
    uint64_t n_blocks;
    uint32_t block_bytes;
    uint32_t n_levels;
    uint64_t words_per_level[DSR_MAX_LEVELS];
    uint64_t bitmap_words;
    uint64_t off_free_bm;
    uint64_t off_alloc_bm;
    uint64_t off_active_bm;
    uint64_t off_obj;        /* uint64[n_blocks]: bit s set iff slot s is free */
    uint64_t off_type;       /* uint8[n_blocks]: type of an allocated block */
    uint64_t off_data;       /* n_blocks * block_bytes of SOA data */
    uint64_t arena_bytes_used;
    uint32_t n_types;
    uint32_t capacity[DSR_MAX_TYPES];
    uint32_t n_fields[DSR_MAX_TYPES];
    uint32_t field_bytes[DSR_MAX_TYPES][DSR_MAX_FIELDS];
    uint32_t field_offset[DSR_MAX_TYPES][DSR_MAX_FIELDS]; /* byte offset of field f's SOA array in a block */
    uint32_t fanout;         /* bits used per bitmap word: 64, 32 or 16 */
    uint32_t pad_;
} dsr_layout;

/* Built-in do-all methods (dsr_parallel_do). Application methods are listed
 * in dsr_apps.h. */
enum {
    DSR_METHOD_COUNT = 1,      /* args: dsr_count_args. Counts visited objects. */
    DSR_METHOD_STREAM_ADD = 2, /* args: none. Field f += field f+1 (32-bit ints), last field += 1. */
    DSR_METHOD_DELETE_IF = 3,  /* args: dsr_delete_if_args. Deletes `this` when field0 mod m == r. */
    DSR_METHOD_CLONE = 4       /* args: dsr_clone_args. Creates a copy of `this` as type dst_type. */
};
typedef struct { unsigned long long* counter_dev; } dsr_count_args;
typedef struct { int32_t modulus; int32_t residue; } dsr_delete_if_args;
typedef struct { int32_t dst_type; int32_t add; } dsr_clone_args;

/* Size in bytes of a heap arena for the given types that yields at least
 * n_blocks blocks. Host-only, no CUDA call. */
int dsr_heap_bytes_for_blocks(const dsr_type_desc* types, int n_types, uint64_t n_blocks,
                              const dsr_tuning* tune, size_t* out_bytes);

/* The layout a heap of n_blocks blocks would have (block geometry, slot
 * capacities, field offsets, metadata offsets). Host-only, no CUDA call. */
int dsr_heap_plan(const dsr_type_desc* types, int n_types, uint64_t n_blocks, const dsr_tuning* tune,
                  dsr_layout* out);

/* Create a heap inside a caller-owned device arena of heap_bytes bytes
 * (256-byte aligned). Carves metadata and M equal-size blocks from the
 * arena, and queues on `stream` the kernel that marks every block free.
 * Block geometry follows Section 2: the smallest type gets cap_min slots per
 * block, which fixes the block size in bytes; every other type gets
 * floor(cap_min * size_min / size_T) slots (at least 1, at most 64). The
 * arena must outlive the heap. Returns DSR_E_INVALID for bad descriptors,
 * DSR_E_OOM if the arena holds no block. */
int dsr_heap_create(const dsr_type_desc* types, int n_types, void* arena_dev, size_t heap_bytes,
                    const dsr_tuning* tune, void* stream, dsr_heap** out);

/* Subtypes (Section 1: class inheritance without wasted memory).
 * base[t] is the direct base type of type t, or -1. A base must be declared
 * before its subtypes (base[t] < t), and a subtype's first fields are its
 * base's fields, with the same sizes, in the same order (so field index f
 * names the same field in a base and in all its subtypes). A subtype has its
 * own blocks, laid out for its own size (its capacity follows from its own
 * fields, not the largest type of the hierarchy). After dsr_heap_set_bases,
 * a do-all over type t (dsr_parallel_do, dsr_doall_scan / dsr_doall_run)
 * visits the live objects of t and of all its transitive subtypes, and the
 * method sees each object's concrete type; dsr_heap_dump and dsr_heap_hash
 * still cover exactly one type. Host-only, no CUDA call; call it before the
 * heap's first do-all (it takes effect in kernels queued after it).
 * dsr_type_tree checks base[] against the descriptors alone and writes
 * sub_out[t], the bit mask of the types a do-all over t visits.
 * DSR_E_INVALID for a base index out of range or after its subtype, or a
 * subtype whose leading fields do not match its base's. */
int dsr_type_tree(const dsr_type_desc* types, int n_types, const int* base, uint32_t* sub_out);
int dsr_heap_set_bases(dsr_heap* heap, const int* base);

/* Free the host handle. Does not touch the arena. */
int dsr_heap_destroy(dsr_heap* heap);

/* Queue a reset of every block to free and clear the error bits. */
int dsr_heap_reset(dsr_heap* heap, void* stream);

/* Layout of the arena (host-only). */
int dsr_heap_layout(const dsr_heap* heap, dsr_layout* out);

/* Device view of the heap: copies sizeof(dsr_dev_heap) bytes (see
 * dsr_device.cuh) into `out`, which a caller passes by value to its own
 * kernels that call dsr_new / dsr_delete. out_bytes must be at least
 * dsr_dev_heap_size(). */
size_t dsr_dev_heap_size(void);
int dsr_heap_device_view(const dsr_heap* heap, void* out, size_t out_bytes);

/* Statistics of a quiescent heap. Queues a reduction over the bitmaps on
 * `stream` and SYNCHRONISES that stream. */
int dsr_heap_stats(dsr_heap* heap, void* stream, dsr_stats* out);

/* Parallel do-all (Section 2.3, Fig. 4): run `method` on every object of
 * `type` that is live when the call starts. Queues (1) a scan of the
 * allocated[type] bitmap that compacts the allocated blocks, with a snapshot
 * of their occupied slots, into the block list R, and (2) the method kernel,
 * in which the threads of each listed block take its slots in order. Objects
 * created while the do-all runs are not visited; a method may delete `this`,
 * or objects of a type other than `type`. args (host memory, args_bytes
 * bytes) is copied into the launch. */
int dsr_parallel_do(dsr_heap* heap, int type, int method, const void* args, size_t args_bytes,
                    void* stream);

/* The two halves of dsr_parallel_do, for callers that time or overlap them:
 * dsr_doall_scan queues steps 1 and 2 of Fig. 4 (the list R of allocated
 * blocks of `type` with their occupied-slot snapshots); dsr_doall_run queues
 * the method kernel over that list. Every dsr_doall_scan must be followed by
 * exactly one dsr_doall_run of the same type on the same stream before the
 * next scan of this heap; the run resets R. */
int dsr_doall_scan(dsr_heap* heap, int type, void* stream);
int dsr_doall_run(dsr_heap* heap, int type, int method, const void* args, size_t args_bytes, void* stream);

/* Write every live object of `type` to out_dev as rows of
 * (32-bit field words..., handle low word, handle high word); an 8-byte
 * field takes two words (low first). Row width = dsr_row_words(type).
 * *count_dev (device uint64) receives the number of objects; rows beyond
 * `cap` are dropped and DSR_ERR_CAPACITY is raised. Row order is arbitrary. */
int dsr_heap_dump(dsr_heap* heap, int type, void* out_dev, uint64_t cap, void* count_dev, void* stream);
int dsr_row_words(const dsr_heap* heap, int type);

/* Order-independent state hash of the live objects of `type`, added to the
 * device uint64 at hash_dev (zero it first). Object hash: h0 = mix64(type +
 * G), h_{i+1} = mix64((h_i ^ w_i) + G) over its 32-bit field words, with
 * mix64 the SplitMix64 finalizer and G = 0x9E3779B97F4A7C15; the state hash
 * is the sum of object hashes modulo 2^64. */
int dsr_heap_hash(dsr_heap* heap, int type, void* hash_dev, void* stream);

/* Event counters (DSR_CTR_* order) summed over SMs: out[DSR_CTR_COUNT]. Synchronises
 * `stream`. */
int dsr_heap_counters(dsr_heap* heap, void* stream, uint64_t* out);

/* Fault injection: the next n slow-path allocations (new block needed) fail
 * as if the heap were full. Queued on `stream`. */
int dsr_heap_inject_oom(dsr_heap* heap, uint32_t n, void* stream);

/* ---- heap groups -----------------------------------------------------------
 * A group carves heaps with the same type descriptors and tuning out of one
 * caller-owned arena and runs do-alls over all of its heaps in single kernel
 * launches (no counterpart in the paper, which runs one heap; this is the
 * batched form: many independent simulations, each with its own heap, so an
 * instance that runs out of memory does not touch the others and a finished
 * instance returns its bytes at once). A group do-all is one fused scan over
 * every heap's allocated[T] bitmap (each listed block tagged with its heap
 * index) and one method kernel over the combined list.
 *   max_heaps   number of heap slots (indices 0 .. max_heaps-1).
 * The arena holds the group's tables and lists first; heaps are placed in the
 * rest, first fit by bytes. */
typedef struct dsr_group dsr_group;
int dsr_group_create(const dsr_type_desc* types, int n_types, void* arena_dev, size_t arena_bytes, int max_heaps,
                     const dsr_tuning* tune, void* stream, dsr_group** out);
/* A group of other types in the same arena as `with` (no counterpart in the
 * paper): its tables and heaps are carved first fit from the free bytes that
 * every group of that arena draws on, so groups of different applications
 * share one pool of memory instead of fixed parts of it. The arena stays
 * owned by the caller and must outlive every group in it; the groups may be
 * destroyed in any order (a destroyed group's bytes return to the pool).
 * Calls on groups of one arena must not run concurrently on the host. */
int dsr_group_create_shared(const dsr_type_desc* types, int n_types, dsr_group* with, int max_heaps,
                            const dsr_tuning* tune, void* stream, dsr_group** out);
int dsr_group_destroy(dsr_group* g);
/* Carve a heap of at least n_blocks blocks plus extra_bytes of caller scratch
 * (256-byte aligned, returned in *extra_dev) and queue its reset on `stream`.
 * Returns DSR_E_OOM when no free range of the arena is large enough (the
 * group is unchanged). The heap handle stays owned by the group. */
int dsr_group_add_heap(dsr_group* g, uint64_t n_blocks, size_t extra_bytes, void* stream, int* index_out,
                       dsr_heap** heap_out, void** extra_dev_out);
/* Return a heap's bytes to the arena. Work queued on the heap must have
 * finished, or be ordered before any later use of the bytes on one stream. */
int dsr_group_remove_heap(dsr_group* g, int index);
/* Bytes a heap of n_blocks blocks plus extra_bytes takes in a group arena. */
int dsr_group_heap_bytes(const dsr_group* g, uint64_t n_blocks, size_t extra_bytes, size_t* out);
/* Free bytes of the arena (shared by every group in it), and the largest free range. */
int dsr_group_free_bytes(const dsr_group* g, size_t* total_free, size_t* largest_free);
int dsr_group_heap_count(const dsr_group* g);
/* Builds compiled with -DDSR_DEVICE_CHECKS check indices and handles on the
 * device; a failed check sets DSR_ERR_CHECK (32) and records the first
 * failure as (code << 48 | value). These calls read the group's and a heap's
 * record (both are 0 in ordinary builds). Synchronous. */
int dsr_group_check_record(dsr_group* g, uint32_t* err_out, uint64_t* record_out);
int dsr_heap_check_record(dsr_heap* heap, uint32_t* err_out, uint64_t* record_out);
/* Group do-all with a built-in method (DSR_METHOD_COUNT). */
int dsr_group_parallel_do(dsr_group* g, int type, int method, const void* args, size_t args_bytes, void* stream);

/* ---- BitmapAlloc: the comparison allocator of Section 4 -------------------
 * "Allocates objects in a large array and uses a bitmap to find empty
 * slots": per type, an array of capacity[T] objects stored as structs (AOS)
 * and a flat bitmap with one bit per slot; no blocks, no bitmap hierarchy.
 * No counterpart in the paper's interface; it exists to compare against.
 * capacity[T] must be a positive multiple of 64. Device code uses the
 * dsr_new / dsr_delete / dsr_field overloads on dsr_bm_dev
 * (paper_1809_07444_gb300/csrc/dsr_bitmap_alloc.cuh). Handles are
 * (type << 40) | slot. Errors as for dsr heaps. */
typedef struct dsr_bm_heap dsr_bm_heap;
int dsr_bm_heap_bytes(const dsr_type_desc* types, int n_types, const uint64_t* capacity, size_t* out);
int dsr_bm_heap_create(const dsr_type_desc* types, int n_types, const uint64_t* capacity, void* arena_dev,
                       size_t arena_bytes, void* stream, dsr_bm_heap** out);
int dsr_bm_heap_destroy(dsr_bm_heap* heap);
/* live_out[T] = objects of type T; *err_out = sticky DSR_ERR_* bits (synchronises). */
int dsr_bm_heap_stats(dsr_bm_heap* heap, void* stream, uint64_t* live_out, uint32_t* err_out);
/* The object-state hash of dsr_heap_hash over the live objects of `type`
 * (types with 4-byte fields only). */
int dsr_bm_heap_hash(dsr_bm_heap* heap, int type, void* hash_dev, void* stream);
int dsr_bm_heap_counters(dsr_bm_heap* heap, void* stream, uint64_t* out);

/* Text for a status code; the CUDA error of the last DSR_E_CUDA. */
const char* dsr_status_string(int status);
const char* dsr_last_cuda_error(void);

/* Microbenchmark kernels (no counterpart in the paper; they measure the two
 * halves of the hot path separately).
 * dsr_bench_alloc: n_threads threads each create one object of type
 * (mix(seed, tid) mod n_types_used) and write tid into its field 0; the
 * handles go to refs_dev (uint64[n_threads], DSR_NULL on failure).
 * dsr_bench_free: deletes every non-null handle of refs_dev. */
int dsr_bench_alloc(dsr_heap* heap, uint64_t n_threads, int n_types_used, uint64_t seed, void* refs_dev,
                    void* stream);
int dsr_bench_free(dsr_heap* heap, uint64_t n_threads, const void* refs_dev, void* stream);
/* dsr_bench_churn: a mixed kernel over the handles of dsr_bench_alloc. Thread
 * i with mix(seed, i) odd (half of them) deletes refs_dev[i] and creates a
 * replacement of type (mix(seed + 1, i) mod n_types_used) holding i in field
 * 0, so deletes and creates of many warps run interleaved. *n_replaced_dev
 * (uint64, device, caller-zeroed) receives the number of replacements. */
int dsr_bench_churn(dsr_heap* heap, uint64_t n_threads, int n_types_used, uint64_t seed, void* refs_dev,
                    void* n_replaced_dev, void* stream);
/* dsr_bench_fma: an FP32 FMA throughput probe, the ALU ceiling of the n-body
 * force kernel. Every thread runs 8 independent FMA chains of `iters` steps
 * and writes one float to out_dev[thread]; the grid is `ctas` x 256 threads.
 * FLOPs = ctas * 256 * 8 * iters * 2. */
int dsr_bench_fma(float* out_dev, int ctas, int iters, void* stream);
/* dsr_bench_atomics: an L2 atomic throughput probe, the ceiling of the
 * allocator's bitmap traffic. One thread per 64-bit word of words_dev
 * (n_words, device), each doing `iters` atomics on its own word: alternating
 * atomicOr and atomicAnd of one bit; with_return = 0 discards the results
 * (reductions), 1 uses them (each waits for the previous). Atomics =
 * n_words * iters. */
int dsr_bench_atomics(void* words_dev, uint64_t n_words, int iters, int with_return, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DSR_H */
