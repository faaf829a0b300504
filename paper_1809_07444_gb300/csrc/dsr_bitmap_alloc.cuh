// BitmapAlloc: the comparison allocator of Section 4 ("allocates objects in
// a large array and uses a bitmap to find empty slots"). Each type has its
// own array of `cap` objects stored as structs (AOS: an object's fields are
// contiguous) and a flat bitmap with one bit per slot (set = the slot holds
// an object). There is no block structure and no bitmap hierarchy.
//
// The device API mirrors the dsr heap's (dsr_new / dsr_delete / dsr_field
// overloads on the heap type), so the same application rules run on both
// allocators. Allocation is warp-aggregated the same way (one leader per
// (heap, type) group), so the comparison isolates the data layout and the
// search structure. A do-all lists the non-zero bitmap words (one entry per
// 64 slots) and runs one thread per slot.
#pragma once

#include "dsr_internal.cuh"

#define DSR_BM_SLOT_BITS 40  // handle = (type << 40) | slot

struct dsr_bm_dev {
    uint8_t* data[DSR_MAX_TYPES];  // cap[T] objects of obj_bytes[T] bytes
    dsr_u64* used[DSR_MAX_TYPES];  // cap[T] / 64 words, bit set = slot in use
    dsr_u64 cap[DSR_MAX_TYPES];    // slots, a multiple of 64
    uint32_t obj_bytes[DSR_MAX_TYPES];
    uint16_t foff[DSR_MAX_TYPES][DSR_MAX_FIELDS];  // field offsets inside an object
    int32_t n_types;
    uint32_t* err;
    dsr_u64* dbg;
    dsr_u64* ctr;        // [DSR_CTR_SLOTS][DSR_CTR_COUNT] event counters
    uint32_t* R_word;    // do-all list: bitmap word index
    dsr_u64* R_mask;     // do-all list: slots in use in the snapshot
    uint32_t* R_count;
    uint32_t* R_done;
};

template <class F>
__device__ __forceinline__ F* dsr_field(const dsr_bm_dev& H, int T, dsr_ref r, int f) {
    const dsr_u64 slot = r & ((1ull << DSR_BM_SLOT_BITS) - 1);
    return reinterpret_cast<F*>(H.data[T] + slot * H.obj_bytes[T] + H.foff[T][f]);
}

/* new T: lanes asking for the same type of the same heap are served by one
 * leader, which probes bitmap words linearly from a hashed start and takes
 * free bits of a word with atomicOr. When another leader took the bits it
 * chose, it retries the same word with the value the atomic returned
 * (bounded); it moves on only from a word it saw full. DSR_NULL (and
 * DSR_ERR_OOM) once a sweep has seen every word of the type full in a row. */
__device__ inline dsr_ref dsr_new(const dsr_bm_dev& H, int T) {
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, (dsr_u64)reinterpret_cast<uintptr_t>(H.used[0]) | (dsr_u64)T);
    const unsigned lane = dsr_lane();
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1));
    const int need = __popc(peers);
    const dsr_u64 nw = H.cap[T] >> 6;
    const unsigned hint = dsr_hash32((blockIdx.x * 0x9E3779B1u) ^ ((threadIdx.x >> 5) * 0x85EBCA77u) ^ (unsigned)T);
    dsr_u64 word = __umulhi(hint, (unsigned)nw);
    dsr_ref mine = DSR_NULL;
    int served = 0;
    while (served < need) {
        dsr_u64 base = 0, bits = 0;
        uint32_t st = 0;
        if ((int)lane == leader) {
            dsr_u64 full_run = 0;  // consecutive words seen full
            for (unsigned a = 0;; ++a) {
                if (full_run > nw || a >= DSR_ALLOC_CAP) {
                    st = full_run > nw ? DSR_ERR_OOM : DSR_ERR_RETRY;
                    atomicOr(H.err, st);
                    break;
                }
                dsr_u64* w = H.used[T] + word;
                dsr_u64 snap = dsr_ld_relaxed(w);
                for (int r = 0; r < 64 && snap != ~0ull && !bits; ++r) {
                    const dsr_u64 want = dsr_lowest_bits(~snap, need - served);
                    const dsr_u64 prev = atomicOr(w, want);
                    bits = want & ~prev;
                    snap = prev | want;
                }
                if (bits) {
                    base = word << 6;
                    break;
                }
                full_run = snap == ~0ull ? full_run + 1 : 0;
                word = word + 1 == nw ? 0 : word + 1;
            }
            if (!st) dsr_count(H.ctr, DSR_CTR_ALLOCS, (dsr_u64)__popcll(bits));
        }
        base = __shfl_sync(peers, base, leader);
        bits = __shfl_sync(peers, bits, leader);
        st = __shfl_sync(peers, st, leader);
        if (st) break;
        const int n = __popcll(bits);
        if (rank >= served && rank < served + n)
            mine = ((dsr_u64)T << DSR_BM_SLOT_BITS) | (base + (dsr_u64)dsr_nth_bit(bits, rank - served));
        served += n;
    }
    return mine;
}
// The placement hint of dsr_new has no counterpart in the comparator.
__device__ inline dsr_ref dsr_new(const dsr_bm_dev& H, int T, dsr_ref) { return dsr_new(H, T); }

/* delete: lanes freeing slots of one bitmap word of one heap are combined
 * into one atomicAnd. */
__device__ inline void dsr_delete(const dsr_bm_dev& H, dsr_ref r) {
    if (r == DSR_NULL) return;
    const unsigned act = __activemask();
    const int T = (int)(r >> DSR_BM_SLOT_BITS);
    const dsr_u64 slot = r & ((1ull << DSR_BM_SLOT_BITS) - 1);
    const dsr_u64 key = r >> 6;  // type and word
    const unsigned peers =
        __match_any_sync(act, key) & __match_any_sync(act, (dsr_u64)reinterpret_cast<uintptr_t>(H.used[0]));
    const unsigned s = (unsigned)(slot & 63);
    const unsigned lo = __reduce_or_sync(peers, s < 32 ? (1u << s) : 0u);
    const unsigned hi = __reduce_or_sync(peers, s >= 32 ? (1u << (s - 32)) : 0u);
    if ((int)dsr_lane() != __ffs(peers) - 1) return;
    if (T >= H.n_types || slot >= H.cap[T]) {
        atomicOr(H.err, DSR_ERR_BAD_HANDLE);
        return;
    }
    const dsr_u64 bits = ((dsr_u64)hi << 32) | lo;
    const dsr_u64 prev = atomicAnd(H.used[T] + (slot >> 6), ~bits);
    if ((prev & bits) != bits) atomicOr(H.err, DSR_ERR_DOUBLE_FREE);
    dsr_count(H.ctr, DSR_CTR_FREES, (dsr_u64)__popcll(bits));
}

/* Optional end-of-do-all hook, as for dsr heaps: Method::finish(H, T, args)
 * runs once, in the last CTA. */
template <class M>
__device__ __forceinline__ auto dsr_bm_call_finish(const dsr_bm_dev& H, int T, const typename M::Args& a, int)
    -> decltype(M::finish(H, T, a), void()) {
    M::finish(H, T, a);
}
template <class M>
__device__ __forceinline__ void dsr_bm_call_finish(const dsr_bm_dev&, int, const typename M::Args&, long) {}

/* Method kernel of a do-all over type T: 64 threads per listed bitmap word;
 * a slot runs the method iff it was in use in the scan's snapshot. keep_list
 * as in dsr_doall_kernel. */
template <class Method>
__global__ void dsr_bm_doall_kernel(const __grid_constant__ dsr_bm_dev H, int T,
                                    const __grid_constant__ typename Method::Args args, int keep_list) {
    const dsr_u64 total = (dsr_u64)(*(volatile uint32_t*)H.R_count) << 6;
    const dsr_u64 stride = (dsr_u64)gridDim.x * blockDim.x;
    for (dsr_u64 g = (dsr_u64)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        __syncwarp();  // warp-uniform loop, as in dsr_doall_kernel
        const dsr_u64 i = g >> 6;
        const unsigned s = (unsigned)(g & 63);
        const dsr_u64 mask = H.R_mask[i];  // loaded together with the word index
        const dsr_u64 word = H.R_word[i];
        if ((mask >> s) & 1ull) Method::run(H, T, args, ((dsr_u64)T << DSR_BM_SLOT_BITS) | ((word << 6) | s));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(H.R_done, 1u) == gridDim.x - 1) {
            if (!keep_list) *(volatile uint32_t*)H.R_count = 0;
            *(volatile uint32_t*)H.R_done = 0;
            __threadfence();
            dsr_bm_call_finish<Method>(H, T, args, 0);
        }
    }
}

// Host side.
struct dsr_bm_heap {
    dsr_bm_dev dev;
    int n_types;
    uint32_t n_fields[DSR_MAX_TYPES];
    uint32_t field_bytes[DSR_MAX_TYPES][DSR_MAX_FIELDS];
    uint8_t* arena;
    int sm_count;
};
void dsr__bm_launch_scan(const dsr_bm_heap* h, int type, cudaStream_t s, unsigned visits_per_object);
int dsr__bm_grid(const dsr_bm_heap* h, const void* kernel, int threads);

template <class M>
int dsr__bm_doall(dsr_bm_heap* h, int type, const typename M::Args& args, cudaStream_t s, bool with_scan = true,
                  int reuse = 0) {
    if (type < 0 || type >= h->n_types) return DSR_E_INVALID;
    if (with_scan) dsr__bm_launch_scan(h, type, s, 1u + (unsigned)reuse);
    const int threads = 256;
    const int grid = dsr__bm_grid(h, (const void*)dsr_bm_doall_kernel<M>, threads);
    dsr_bm_doall_kernel<M><<<grid, threads, 0, s>>>(h->dev, type, args, reuse > 0 ? 1 : 0);
    return dsr__check_launch("dsr_bm_doall_kernel");
}
