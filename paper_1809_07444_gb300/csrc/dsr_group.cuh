// Host-side internals of heap groups, shared by the group and the batched
// applications.
#pragma once

#include <map>
#include <memory>
#include <vector>

#include "dsr_internal.cuh"

// The bytes of one caller-owned arena, handed out first fit. Every group
// carved from the arena holds the pool (dsr_group_create makes one,
// dsr_group_create_shared joins another group's); its tables, its heaps and
// the application's instance tables all come from it.
struct dsr_pool {
    uint8_t* arena;
    size_t bytes;
    std::map<size_t, size_t> free_ranges;  // offset -> bytes
};
// First fit of `need` bytes (a multiple of 1024); false if no range is large enough.
bool dsr__pool_take(dsr_pool& p, size_t need, size_t* off);
// Return a range, merged with its free neighbours.
void dsr__pool_give(dsr_pool& p, size_t off, size_t size);

struct dsr_group {
    std::shared_ptr<dsr_pool> pool;
    uint8_t* arena;                        // pool->arena
    size_t tables_off, tables_bytes;       // this group's tables and lists in the arena
    int max_heaps;
    uint64_t max_chunks;
    int n_types;
    std::vector<dsr_type_desc> types;
    std::vector<std::vector<int>> fields;
    dsr_tuning tune;
    int device;
    int sm_count;
    std::vector<dsr_heap*> heaps;          // slot -> heap (nullptr = free slot)
    std::vector<size_t> offsets, sizes;    // slot -> range in the arena
    std::vector<dsr_dev_heap> views;       // host copies of the device views
    std::vector<uint32_t> chunk_heap_h, chunk_base_h;
    uint32_t n_chunks = 0;
    uint64_t epoch = 0;                    // bumped whenever the set of heaps changes
    dsr_dev_heap* heaps_d;
    uint32_t* chunk_heap_d;
    uint32_t* chunk_base_d;
    dsr_group_dev dev;
};

// Bytes for an application's own tables from the group's pool (a multiple
// of 1024, 1024-aligned); DSR_E_OOM if none is free. Give them back before
// the group is destroyed.
int dsr__group_take_bytes(dsr_group* g, size_t bytes, void** out);
void dsr__group_give_bytes(dsr_group* g, void* p, size_t bytes);

void dsr__group_launch_scan(const dsr_group* g, int type, cudaStream_t s, unsigned visits_per_object = 1);
int dsr__group_grid(const dsr_group* g, const void* kernel, int threads);

// Slots of a block of type T covered per listed block (log2): 5 for
// capacities up to 32, else 6; the same for every heap of a group.
inline unsigned dsr__group_span(const dsr_group* g, int type) {
    dsr_layout L;
    dsr_heap_plan(g->types.data(), g->n_types, 1, &g->tune, &L);
    return L.capacity[type] <= 32 ? 5u : 6u;
}

// A group do-all: fused scan over every heap, then the method kernel.
// with_scan / reuse as in dsr__doall: reuse > 0 keeps the block list for
// that many following do-alls over the same live set, which pass
// with_scan = false.
template <class M>
int dsr__group_doall(dsr_group* g, int type, const typename M::Args& args, cudaStream_t s, bool with_scan = true,
                     int reuse = 0) {
    if (type < 0 || type >= g->n_types) return DSR_E_INVALID;
    if (with_scan) dsr__group_launch_scan(g, type, s, 1u + (unsigned)reuse);
    const int threads = g->tune.threads > 0 ? g->tune.threads : 256;
    if (threads <= 256) {
        const int grid = dsr__group_grid(g, (const void*)dsr_group_doall_kernel_256<M>, threads);
        dsr_group_doall_kernel_256<M><<<grid, threads, 0, s>>>(g->dev, type, dsr__group_span(g, type), args,
                                                               reuse > 0 ? 1 : 0);
    } else {
        const int grid = dsr__group_grid(g, (const void*)dsr_group_doall_kernel<M>, threads);
        dsr_group_doall_kernel<M><<<grid, threads, 0, s>>>(g->dev, type, dsr__group_span(g, type), args,
                                                           reuse > 0 ? 1 : 0);
    }
    return dsr__check_launch("dsr_group_doall_kernel");
}
