// Heap groups: many heaps carved from one arena, with do-alls that cover all
// of them in single launches (one fused scan, one method kernel).
#include <map>
#include <new>
#include <vector>

#include "dsr_group.cuh"

// ---------------------------------------------------------------------------
// fused scan: as the single-heap scan, over chunks of 256 block ids of any
// heap of the group; every listed block is tagged with its heap index
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_group_scan(const __grid_constant__ dsr_group_dev G, int T,
                                                    unsigned visits_mult) {
    __shared__ unsigned warp_n[8];
    __shared__ unsigned run_base;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t c = blockIdx.x; c < G.n_chunks; c += gridDim.x) {
        const uint32_t h = G.chunk_heap[c];
        const bool hok = dsr_check(h < G.n_slots, G.err, G.dbg, 1, c);
        const dsr_dev_heap& H = G.heaps[hok ? h : 0];
        const dsr_u64 b = (dsr_u64)G.chunk_base[c] + threadIdx.x;
        const unsigned fsh = H.alloc_bm[T].shift;
        const bool set = hok && b < H.M && ((H.alloc_bm[T].lvl[0][b >> fsh] >> (b & ((1u << fsh) - 1))) & 1ull);
        const unsigned ballot = __ballot_sync(0xFFFFFFFFu, set);
        if (lane == 0) warp_n[warp] = __popc(ballot);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned total = 0;
            for (int w = 0; w < 8; ++w) {
                const unsigned n = warp_n[w];
                warp_n[w] = total;
                total += n;
            }
            run_base = total ? atomicAdd(G.R_count, total) : 0;
        }
        __syncthreads();
        unsigned objs = 0;
        const unsigned k = run_base + warp_n[warp] + __popc(ballot & ((1u << lane) - 1));
        if (set && dsr_check(k < G.R_cap, G.err, G.dbg, 2, k)) {
            const dsr_u64 live = H.valid[T] & ~H.obj[b];
            G.R_heap[k] = h;
            G.R_bid[k] = (uint32_t)b;
            G.R_mask[k] = live;
            objs = __popcll(live);
        }
        objs = __reduce_add_sync(0xFFFFFFFFu, objs);
        if (lane == 0 && objs) dsr_count(H.ctr, DSR_CTR_VISITS, (dsr_u64)objs * visits_mult);
        __syncthreads();
    }
}

// First failed device check of the group (checked builds): err word and record.
extern "C" int dsr_group_check_record(dsr_group* g, uint32_t* err_out, uint64_t* record_out) {
    if (!g) return DSR_E_INVALID;
    uint32_t e32 = 0;
    dsr_u64 rec = 0;
    cudaError_t e = cudaMemcpy(&e32, g->dev.err, 4, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(&rec, g->dev.dbg, 8, cudaMemcpyDeviceToHost);
    if (e) {
        dsr__set_cuda_error(e, "dsr_group_check_record");
        return DSR_E_CUDA;
    }
    if (err_out) *err_out = e32;
    if (record_out) *record_out = rec;
    return DSR_OK;
}

void dsr__group_launch_scan(const dsr_group* g, int type, cudaStream_t s, unsigned visits_per_object) {
    if (g->n_chunks == 0) return;
    unsigned ctas = g->n_chunks;
    const unsigned cap = (unsigned)g->sm_count * 8;
    if (ctas > cap) ctas = cap;
    k_group_scan<<<ctas, 256, 0, s>>>(g->dev, type, visits_per_object);
}

int dsr__group_grid(const dsr_group* g, const void* kernel, int threads) {
    int per_sm = g->tune.ctas_per_sm;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
    }
    uint64_t grid = (uint64_t)per_sm * g->sm_count;
    const uint64_t work = ((uint64_t)g->n_chunks * 256 * 64 + threads - 1) / threads;
    if (grid > work) grid = work;
    return grid < 1 ? 1 : (int)grid;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Rebuild the chunk table of the heaps in use and upload it.
static int upload_tables(dsr_group* g, cudaStream_t s) {
    g->chunk_heap_h.clear();
    g->chunk_base_h.clear();
    uint32_t slots = 0;
    for (int i = 0; i < g->max_heaps; ++i) {
        if (!g->heaps[i]) continue;
        slots = (uint32_t)i + 1;
        const uint64_t M = g->heaps[i]->layout.n_blocks;
        for (uint64_t b = 0; b < M; b += 256) {
            g->chunk_heap_h.push_back((uint32_t)i);
            g->chunk_base_h.push_back((uint32_t)b);
        }
    }
    g->n_chunks = (uint32_t)g->chunk_heap_h.size();
    if (g->n_chunks > g->max_chunks) return DSR_E_OOM;
    g->dev.n_chunks = g->n_chunks;
    g->dev.n_slots = slots;
    cudaError_t e = cudaSuccess;
    if (g->n_chunks) {
        e = cudaMemcpyAsync(g->chunk_heap_d, g->chunk_heap_h.data(), g->n_chunks * 4, cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemcpyAsync(g->chunk_base_d, g->chunk_base_h.data(), g->n_chunks * 4, cudaMemcpyHostToDevice, s);
    }
    if (!e) e = cudaStreamSynchronize(s);  // the host vectors may change before an async copy reads them
    if (e) {
        dsr__set_cuda_error(e, "dsr_group tables");
        return DSR_E_CUDA;
    }
    ++g->epoch;
    return DSR_OK;
}

bool dsr__pool_take(dsr_pool& p, size_t need, size_t* off) {
    auto it = p.free_ranges.begin();
    for (; it != p.free_ranges.end(); ++it)
        if (it->second >= need) break;
    if (it == p.free_ranges.end()) return false;
    *off = it->first;
    const size_t rest = it->second - need;
    p.free_ranges.erase(it);
    if (rest) p.free_ranges[*off + need] = rest;
    return true;
}

void dsr__pool_give(dsr_pool& p, size_t off, size_t size) {
    auto next = p.free_ranges.lower_bound(off);
    if (next != p.free_ranges.end() && off + size == next->first) {
        size += next->second;
        p.free_ranges.erase(next);
    }
    auto prev = p.free_ranges.lower_bound(off);
    if (prev != p.free_ranges.begin()) {
        --prev;
        if (prev->first + prev->second == off) {
            off = prev->first;
            size += prev->second;
            p.free_ranges.erase(prev);
        }
    }
    p.free_ranges[off] = size;
}

int dsr__group_take_bytes(dsr_group* g, size_t bytes, void** out) {
    size_t off = 0;
    if (!dsr__pool_take(*g->pool, round_up(bytes, 1024), &off)) return DSR_E_OOM;
    *out = g->arena + off;
    return DSR_OK;
}

void dsr__group_give_bytes(dsr_group* g, void* p, size_t bytes) {
    dsr__pool_give(*g->pool, (size_t)(static_cast<uint8_t*>(p) - g->arena), round_up(bytes, 1024));
}

// A group in `pool`: its tables and lists are carved first fit from the pool,
// sized so that the group's heaps could take the whole arena.
static int group_create_in(std::shared_ptr<dsr_pool> pool, const dsr_type_desc* types, int n_types, int max_heaps,
                           const dsr_tuning* tune, void* stream, dsr_group** out) {
    // Smallest heap footprint per block, to size the group's lists.
    size_t one = 0;
    int rc = dsr_heap_bytes_for_blocks(types, n_types, 1, tune, &one);
    if (rc) return rc;
    size_t two = 0;
    rc = dsr_heap_bytes_for_blocks(types, n_types, 1025, tune, &two);
    if (rc) return rc;
    const size_t per_block = (two - one) / 1024;  // marginal bytes of one more block
    const uint64_t max_blocks = pool->bytes / (per_block ? per_block : 1);
    const uint64_t max_chunks = max_blocks / 256 + (uint64_t)max_heaps;
    size_t off = 0;
    const size_t o_heaps = off;
    off = round_up(off + (size_t)max_heaps * sizeof(dsr_dev_heap), 256);
    const size_t o_ch = off;
    off = round_up(off + max_chunks * 4, 256);
    const size_t o_cb = off;
    off = round_up(off + max_chunks * 4, 256);
    const size_t o_rh = off;
    off = round_up(off + max_blocks * 4, 256);
    const size_t o_rb = off;
    off = round_up(off + max_blocks * 4, 256);
    const size_t o_rm = off;
    off = round_up(off + max_blocks * 8, 256);
    const size_t o_cnt = off;
    off = round_up(off + 256, 1024);
    size_t base = 0;
    if (!dsr__pool_take(*pool, off, &base)) return DSR_E_OOM;

    dsr_group* g = new (std::nothrow) dsr_group;
    if (!g) {
        dsr__pool_give(*pool, base, off);
        return DSR_E_OOM;
    }
    uint8_t* a = pool->arena + base;
    g->pool = pool;
    g->arena = pool->arena;
    g->tables_off = base;
    g->tables_bytes = off;
    g->max_heaps = max_heaps;
    g->max_chunks = max_chunks;
    g->n_types = n_types;
    g->types.assign(types, types + n_types);
    for (int t = 0; t < n_types; ++t) {
        g->fields.emplace_back(types[t].field_bytes, types[t].field_bytes + types[t].n_fields);
        g->types[t].field_bytes = nullptr;  // re-pointed below, after the vectors are in place
    }
    for (int t = 0; t < n_types; ++t) g->types[t].field_bytes = g->fields[t].data();
    g->tune = tune ? *tune : dsr_tuning{0, 0, 0, 0};
    g->heaps.assign(max_heaps, nullptr);
    g->offsets.assign(max_heaps, 0);
    g->sizes.assign(max_heaps, 0);
    g->views.assign(max_heaps, dsr_dev_heap{});
    g->heaps_d = reinterpret_cast<dsr_dev_heap*>(a + o_heaps);
    g->chunk_heap_d = reinterpret_cast<uint32_t*>(a + o_ch);
    g->chunk_base_d = reinterpret_cast<uint32_t*>(a + o_cb);
    g->dev.heaps = g->heaps_d;
    g->dev.chunk_heap = g->chunk_heap_d;
    g->dev.chunk_base = g->chunk_base_d;
    g->dev.R_heap = reinterpret_cast<uint32_t*>(a + o_rh);
    g->dev.R_bid = reinterpret_cast<uint32_t*>(a + o_rb);
    g->dev.R_mask = reinterpret_cast<dsr_u64*>(a + o_rm);
    g->dev.R_count = reinterpret_cast<uint32_t*>(a + o_cnt);
    g->dev.R_done = reinterpret_cast<uint32_t*>(a + o_cnt + 4);
    g->dev.err = reinterpret_cast<uint32_t*>(a + o_cnt + 8);
    g->dev.dbg = reinterpret_cast<dsr_u64*>(a + o_cnt + 16);
    g->dev.R_cap = max_blocks;
    cudaError_t e = cudaGetDevice(&g->device);
    if (!e) e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
    if (!e) e = cudaMemsetAsync(a + o_cnt, 0, 256, dsr__stream(stream));
    if (e) {
        dsr__set_cuda_error(e, "dsr_group_create");
        dsr__pool_give(*pool, base, off);
        delete g;
        return DSR_E_CUDA;
    }
    *out = g;
    return DSR_OK;
}

extern "C" int dsr_group_create(const dsr_type_desc* types, int n_types, void* arena_dev, size_t arena_bytes,
                                int max_heaps, const dsr_tuning* tune, void* stream, dsr_group** out) {
    if (!out || !arena_dev || max_heaps < 1 || (reinterpret_cast<uintptr_t>(arena_dev) & 255)) return DSR_E_INVALID;
    *out = nullptr;
    auto pool = std::make_shared<dsr_pool>();
    pool->arena = static_cast<uint8_t*>(arena_dev);
    pool->bytes = arena_bytes / 1024 * 1024;
    if (pool->bytes == 0) return DSR_E_OOM;
    pool->free_ranges[0] = pool->bytes;
    return group_create_in(pool, types, n_types, max_heaps, tune, stream, out);
}

extern "C" int dsr_group_create_shared(const dsr_type_desc* types, int n_types, dsr_group* with, int max_heaps,
                                       const dsr_tuning* tune, void* stream, dsr_group** out) {
    if (!out || !with || max_heaps < 1) return DSR_E_INVALID;
    *out = nullptr;
    return group_create_in(with->pool, types, n_types, max_heaps, tune, stream, out);
}

extern "C" int dsr_group_destroy(dsr_group* g) {
    if (!g) return DSR_E_INVALID;
    for (int i = 0; i < g->max_heaps; ++i) {
        if (!g->heaps[i]) continue;
        dsr_heap_destroy(g->heaps[i]);
        dsr__pool_give(*g->pool, g->offsets[i], g->sizes[i]);  // for the other groups of a shared pool
    }
    dsr__pool_give(*g->pool, g->tables_off, g->tables_bytes);
    delete g;
    return DSR_OK;
}

extern "C" int dsr_group_heap_bytes(const dsr_group* g, uint64_t n_blocks, size_t extra_bytes, size_t* out) {
    if (!g || !out) return DSR_E_INVALID;
    size_t hb = 0;
    int rc = dsr_heap_bytes_for_blocks(g->types.data(), g->n_types, n_blocks, &g->tune, &hb);
    if (rc) return rc;
    *out = round_up(hb, 1024) + round_up(extra_bytes, 1024);
    return DSR_OK;
}

extern "C" int dsr_group_add_heap(dsr_group* g, uint64_t n_blocks, size_t extra_bytes, void* stream, int* index_out,
                                  dsr_heap** heap_out, void** extra_dev_out) {
    if (!g || !index_out || n_blocks == 0) return DSR_E_INVALID;
    int slot = -1;
    for (int i = 0; i < g->max_heaps; ++i)
        if (!g->heaps[i]) {
            slot = i;
            break;
        }
    if (slot < 0) return DSR_E_OOM;
    size_t hb = 0;
    int rc = dsr_heap_bytes_for_blocks(g->types.data(), g->n_types, n_blocks, &g->tune, &hb);
    if (rc) return rc;
    // The heap gets exactly the bytes of n_blocks blocks (so exactly n_blocks
    // blocks); its range is rounded up so that the extra bytes after it stay
    // aligned.
    const size_t need = round_up(hb, 1024) + round_up(extra_bytes, 1024);
    size_t off = 0;
    if (!dsr__pool_take(*g->pool, need, &off)) return DSR_E_OOM;
    dsr_heap* h = nullptr;
    rc = dsr_heap_create(g->types.data(), g->n_types, g->arena + off, hb, &g->tune, stream, &h);
    if (rc) {
        dsr__pool_give(*g->pool, off, need);
        return rc;
    }
    g->heaps[slot] = h;
    g->offsets[slot] = off;
    g->sizes[slot] = need;
    g->views[slot] = h->dev;
    cudaStream_t s = dsr__stream(stream);
    cudaError_t e = cudaMemcpyAsync(g->heaps_d + slot, &g->views[slot], sizeof(dsr_dev_heap), cudaMemcpyHostToDevice, s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_group_add_heap");
        return DSR_E_CUDA;
    }
    rc = upload_tables(g, s);
    if (rc) return rc;
    *index_out = slot;
    if (heap_out) *heap_out = h;
    if (extra_dev_out) *extra_dev_out = g->arena + off + round_up(hb, 1024);
    return DSR_OK;
}

extern "C" int dsr_group_remove_heap(dsr_group* g, int index) {
    if (!g || index < 0 || index >= g->max_heaps || !g->heaps[index]) return DSR_E_INVALID;
    dsr_heap_destroy(g->heaps[index]);
    g->heaps[index] = nullptr;
    dsr__pool_give(*g->pool, g->offsets[index], g->sizes[index]);
    return upload_tables(g, nullptr);
}

extern "C" int dsr_group_free_bytes(const dsr_group* g, size_t* total_free, size_t* largest_free) {
    if (!g) return DSR_E_INVALID;
    size_t t = 0, l = 0;
    for (auto& kv : g->pool->free_ranges) {
        t += kv.second;
        if (kv.second > l) l = kv.second;
    }
    if (total_free) *total_free = t;
    if (largest_free) *largest_free = l;
    return DSR_OK;
}

extern "C" int dsr_group_heap_count(const dsr_group* g) {
    if (!g) return -1;
    int n = 0;
    for (dsr_heap* h : g->heaps) n += h != nullptr;
    return n;
}

namespace {
struct GCount {
    typedef dsr_count_args Args;
    static __device__ void run(const dsr_dev_heap&, int, const Args& a, dsr_ref, uint32_t) {
        const unsigned act = __activemask();
        if (dsr_lane() == (unsigned)(__ffs(act) - 1)) atomicAdd(a.counter_dev, (dsr_u64)__popc(act));
    }
};
}  // namespace

extern "C" int dsr_group_parallel_do(dsr_group* g, int type, int method, const void* args, size_t args_bytes,
                                     void* stream) {
    if (!g || type < 0 || type >= g->n_types) return DSR_E_INVALID;
    if (method != DSR_METHOD_COUNT || !args || args_bytes != sizeof(dsr_count_args)) return DSR_E_INVALID;
    dsr_count_args a;
    memcpy(&a, args, sizeof a);
    return dsr__group_doall<GCount>(g, type, a, dsr__stream(stream));
}
