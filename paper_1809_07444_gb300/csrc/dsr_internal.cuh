// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "dsr.h"
#include "dsr_device.cuh"

struct dsr_heap {
    dsr_dev_heap dev;    // device view, passed by value to every kernel
    dsr_layout layout;
    uint8_t* arena;
    size_t heap_bytes;
    dsr_tuning tune;
    int device;
    int sm_count;
    dsr_u64* stats_dev;  // scratch in the arena header
    uint64_t version = 0;  // bumped when `dev` changes after creation (launches captured in a graph hold a copy)
};

// Arena header (first DSR_HEADER_BYTES bytes of the arena).
#define DSR_HEADER_BYTES 32768u
#define DSR_HDR_ERR 0u
#define DSR_HDR_INJECT 4u
#define DSR_HDR_RCOUNT 8u
#define DSR_HDR_RDONE 12u
#define DSR_HDR_STATS 256u  // dsr_u64[1 + 3 * DSR_MAX_TYPES]
#define DSR_HDR_SLOW 192u   // uint32[DSR_MAX_TYPES] slow paths in flight
#define DSR_HDR_DBG 224u    // dsr_u64 first failed device check + 24 scratch bytes
#define DSR_HDR_CTR 4096u   // dsr_u64[DSR_CTR_SLOTS][DSR_CTR_COUNT] event counters (16 KB)

void dsr__set_cuda_error(cudaError_t e, const char* where);
int dsr__check_launch(const char* where);

inline cudaStream_t dsr__stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Persistent grid for a method kernel: CTAs that fit on the GPU at once,
// capped by the most work a do-all over this heap can list.
int dsr__persistent_grid(const dsr_heap* h, const void* kernel, int threads);
int dsr__scan_grid(const dsr_heap* h, int type);
// True if every field array of `type` starts on a 16-byte boundary within a
// block and the capacity is a multiple of 4 (vector methods may run).
bool dsr__vec4_ok(const dsr_heap* h, int type);
// exact: list the blocks of `type` only, not those of its subtypes.
void dsr__launch_scan(const dsr_heap* h, int type, cudaStream_t s, unsigned visits_per_object = 1, bool exact = false);

// Run a do-all: scan + compaction of allocated[type] into R, then the method
// kernel over the listed blocks.
// ev_scan / ev_run (optional): recorded on s after the scan and after the
// method kernel, for per-phase timing (as external records, so that under
// stream capture they become event-record nodes of the graph). reuse > 0: the block list is kept for
// `reuse` more do-alls over the same live set, and the scan counts each
// listed object 1 + reuse times as visited (the visits those do-alls make).
// exact: visit the objects of `type` only, not those of its subtypes.
template <class M>
int dsr__doall(dsr_heap* h, int type, const typename M::Args& args, cudaStream_t s, bool with_scan = true,
               cudaEvent_t ev_scan = nullptr, cudaEvent_t ev_run = nullptr, int reuse = 0, bool exact = false) {
    if (type < 0 || type >= h->dev.n_types) return DSR_E_INVALID;
    if (with_scan) dsr__launch_scan(h, type, s, 1u + (unsigned)reuse, exact);
    if (ev_scan) cudaEventRecordWithFlags(ev_scan, s, cudaEventRecordExternal);
    // The occupancy-limited grid of this kernel and CTA size is looked up
    // once and cached; a heap whose tuning fixes the CTAs per SM computes its
    // own and leaves the cache alone (other heaps keep the occupancy limit).
    static int grid_cache[17] = {0};
    const int threads = h->tune.threads;
    const bool small = threads <= 256;  // the occupancy-bounded kernel
    const void* kfn = small ? (const void*)dsr_doall_kernel_256<M> : (const void*)dsr_doall_kernel<M>;
    int grid;
    if (h->tune.ctas_per_sm > 0) {
        grid = dsr__persistent_grid(h, kfn, threads);
    } else {
        int& cached = grid_cache[threads / 64];
        if (cached == 0) cached = dsr__persistent_grid(h, kfn, threads);
        grid = cached;
    }
    // Persistent grid: the CTAs that fit on the GPU at once, capped by the
    // work a do-all over this heap can list. (Every CTA ends with one atomic
    // on the completion counter, so a much larger grid costs more in those
    // serialised atomics than it gains in balance.)
    dsr_u64 g64 = (dsr_u64)grid;
    const dsr_u64 cap_grid = (h->dev.M * 64 + threads - 1) / threads;
    if (g64 > cap_grid) g64 = cap_grid;
    int g = (int)g64;
    if ((dsr_u64)g > cap_grid) g = (int)cap_grid;
    if (g < 1) g = 1;
    int rc;
    if constexpr (dsr_has_run4<M>::value) {
        if (dsr__vec4_ok(h, type)) {
            static int vgrid_cache[17] = {0};
            int vgrid;
            if (h->tune.ctas_per_sm > 0) {
                vgrid = dsr__persistent_grid(h, (const void*)dsr_doall_kernel_vec4<M>, threads);
            } else {
                int& cached = vgrid_cache[threads / 64];
                if (cached == 0) cached = dsr__persistent_grid(h, (const void*)dsr_doall_kernel_vec4<M>, threads);
                vgrid = cached;
            }
            int gv = vgrid < g ? vgrid : g;
            dsr_doall_kernel_vec4<M><<<gv, threads, 0, s>>>(h->dev, type, args, reuse > 0 ? 1 : 0);
            rc = dsr__check_launch("dsr_doall_kernel_vec4");
            if (ev_run) cudaEventRecordWithFlags(ev_run, s, cudaEventRecordExternal);
            return rc;
        }
    }
    if (small)
        dsr_doall_kernel_256<M><<<g, threads, 0, s>>>(h->dev, type, args, reuse > 0 ? 1 : 0);
    else
        dsr_doall_kernel<M><<<g, threads, 0, s>>>(h->dev, type, args, reuse > 0 ? 1 : 0);
    rc = dsr__check_launch("dsr_doall_kernel");
    if (ev_run) cudaEventRecordWithFlags(ev_run, s, cudaEventRecordExternal);
    return rc;
}

// Application method dispatch (defined in the application files).
int dsr__gol_method(dsr_heap* h, int type, int method, const void* args, size_t bytes, cudaStream_t s,
                    bool with_scan);
int dsr__wator_method(dsr_heap* h, int type, int method, const void* args, size_t bytes, cudaStream_t s,
                      bool with_scan);
int dsr__nbody_method(dsr_heap* h, int type, int method, const void* args, size_t bytes, cudaStream_t s,
                      bool with_scan);

// SplitMix64 finalizer and the object-state hash (same definition as the
// dsr_heap_hash documentation).
__device__ __forceinline__ dsr_u64 dsr_mix64(dsr_u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
#define DSR_GAMMA 0x9E3779B97F4A7C15ull
__device__ __forceinline__ dsr_u64 dsr_splitmix_at(dsr_u64 s, dsr_u64 n) { return dsr_mix64(s + (n + 1) * DSR_GAMMA); }
// Counter-based draw keyed on (seed, stream, step, cell).
__device__ __forceinline__ dsr_u64 dsr_rand(dsr_u64 seed, dsr_u64 stream, dsr_u64 step, dsr_u64 cell) {
    return dsr_splitmix_at(dsr_splitmix_at(dsr_splitmix_at(seed, stream), step), cell);
}
