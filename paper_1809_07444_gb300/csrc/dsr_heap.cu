// Heap creation, block geometry, the do-all scan, statistics, generic
// methods and the C ABI of dsr.h.
#include <algorithm>
#include <cstdlib>
#include <new>

#include "dsr_internal.cuh"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_cuda_err[256] = "";

void dsr__set_cuda_error(cudaError_t e, const char* where) {
    snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", where, cudaGetErrorString(e));
}

int dsr__check_launch(const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        dsr__set_cuda_error(e, where);
        return DSR_E_CUDA;
    }
    return DSR_OK;
}

extern "C" const char* dsr_last_cuda_error(void) { return g_cuda_err; }

extern "C" const char* dsr_status_string(int s) {
    switch (s) {
        case DSR_OK: return "ok";
        case DSR_E_INVALID: return "invalid argument";
        case DSR_E_OOM: return "arena too small";
        case DSR_E_CUDA: return "CUDA error";
        case DSR_E_DEVICE: return "device-side error";
        case DSR_E_TOO_LARGE: return "size exceeds the entry point's fixed maximum";
        default: return "unknown status";
    }
}

// ---------------------------------------------------------------------------
// geometry (Section 2: equal-size blocks; the smallest type has cap_min
// slots, which fixes the block size; larger types get fewer slots in
// proportion to their size)
// ---------------------------------------------------------------------------
static inline uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

static uint64_t type_bytes(const dsr_layout& L, int t, uint32_t cap) {
    uint64_t off = 0;
    for (uint32_t f = 0; f < L.n_fields[t]; ++f) off += round_up((uint64_t)cap * L.field_bytes[t][f], 8);
    return off;
}

static int geometry(const dsr_type_desc* types, int n_types, const dsr_tuning& tune, dsr_layout* L) {
    if (!types || n_types < 1 || n_types > DSR_MAX_TYPES) return DSR_E_INVALID;
    if (tune.cap_min != 32 && tune.cap_min != 64) return DSR_E_INVALID;
    if (tune.fanout != 16 && tune.fanout != 32 && tune.fanout != 64) return DSR_E_INVALID;
    memset(L, 0, sizeof *L);
    L->fanout = (uint32_t)tune.fanout;
    L->n_types = (uint32_t)n_types;
    uint64_t smin = ~0ull;
    int tmin = 0;
    uint64_t size[DSR_MAX_TYPES];
    for (int t = 0; t < n_types; ++t) {
        const dsr_type_desc& d = types[t];
        if (d.n_fields < 1 || d.n_fields > DSR_MAX_FIELDS || !d.field_bytes) return DSR_E_INVALID;
        L->n_fields[t] = (uint32_t)d.n_fields;
        size[t] = 0;
        for (int f = 0; f < d.n_fields; ++f) {
            if (d.field_bytes[f] != 4 && d.field_bytes[f] != 8) return DSR_E_INVALID;
            L->field_bytes[t][f] = (uint32_t)d.field_bytes[f];
            size[t] += (uint64_t)d.field_bytes[f];
        }
        if (size[t] < smin) {
            smin = size[t];
            tmin = t;
        }
    }
    const uint64_t block_bytes = round_up(type_bytes(*L, tmin, (uint32_t)tune.cap_min), 128);
    L->block_bytes = (uint32_t)block_bytes;
    for (int t = 0; t < n_types; ++t) {
        uint64_t c = (uint64_t)tune.cap_min * smin / size[t];
        if (c > 64) c = 64;
        if (c < 1) c = 1;
        while (c > 1 && type_bytes(*L, t, (uint32_t)c) > block_bytes) --c;
        L->capacity[t] = (uint32_t)c;
        uint64_t off = 0;
        for (uint32_t f = 0; f < L->n_fields[t]; ++f) {
            L->field_offset[t][f] = (uint32_t)off;
            off += round_up(c * L->field_bytes[t][f], 8);
        }
    }
    return DSR_OK;
}

// Offsets of every metadata array for M blocks; returns the arena bytes used,
// or UINT64_MAX if the bitmaps would need more than DSR_MAX_LEVELS levels.
static uint64_t place(dsr_layout* L, uint64_t M) {
    L->n_blocks = M;
    const uint64_t f = L->fanout;
    uint64_t n = M;
    int lv = 0;
    uint64_t words = 0;
    for (;;) {
        if (lv == DSR_MAX_LEVELS) return ~0ull;
        L->words_per_level[lv] = (n + f - 1) / f;
        words += L->words_per_level[lv];
        ++lv;
        if (n <= f) break;
        n = (n + f - 1) / f;
    }
    L->n_levels = (uint32_t)lv;
    L->bitmap_words = words;
    const uint64_t T = L->n_types;
    uint64_t off = DSR_HEADER_BYTES;
    L->off_free_bm = off;
    off += words * 8;
    L->off_alloc_bm = off;
    off += T * words * 8;
    L->off_active_bm = off;
    off += T * words * 8;
    off = round_up(off, 256);
    L->off_obj = off;
    off += M * 8;
    off = round_up(off, 256);
    uint64_t off_rmask = off;
    off += M * 8;
    off = round_up(off, 256);
    uint64_t off_rbid = off;
    off += M * 4;
    off = round_up(off, 256);
    L->off_type = off;
    off += M;
    off = round_up(off, 1024);
    L->off_data = off;
    off += M * L->block_bytes;
    L->arena_bytes_used = off;
    (void)off_rmask;
    (void)off_rbid;
    return off;
}

static uint64_t off_rmask(const dsr_layout& L) { return round_up(L.off_obj + L.n_blocks * 8, 256); }
static uint64_t off_rbid(const dsr_layout& L) { return round_up(off_rmask(L) + L.n_blocks * 8, 256); }

static dsr_tuning resolve_tuning(const dsr_tuning* t) {
    dsr_tuning r{64, 256, 0, 64};
    if (t) {
        if (t->cap_min) r.cap_min = t->cap_min;
        if (t->threads) r.threads = t->threads;
        r.ctas_per_sm = t->ctas_per_sm;
        if (t->fanout) r.fanout = t->fanout;
    }
    return r;
}

extern "C" int dsr_heap_bytes_for_blocks(const dsr_type_desc* types, int n_types, uint64_t n_blocks,
                                         const dsr_tuning* tune, size_t* out_bytes) {
    if (!out_bytes || n_blocks == 0 || n_blocks > 0xFFFFFFFFull) return DSR_E_INVALID;
    dsr_layout L;
    int rc = geometry(types, n_types, resolve_tuning(tune), &L);
    if (rc) return rc;
    const uint64_t bytes = place(&L, n_blocks);
    if (bytes == ~0ull) return DSR_E_INVALID;
    *out_bytes = (size_t)bytes;
    return DSR_OK;
}

extern "C" int dsr_heap_plan(const dsr_type_desc* types, int n_types, uint64_t n_blocks, const dsr_tuning* tune,
                             dsr_layout* out) {
    if (!out || n_blocks == 0 || n_blocks > 0xFFFFFFFFull) return DSR_E_INVALID;
    dsr_layout L;
    int rc = geometry(types, n_types, resolve_tuning(tune), &L);
    if (rc) return rc;
    if (place(&L, n_blocks) == ~0ull) return DSR_E_INVALID;
    *out = L;
    return DSR_OK;
}

// ---------------------------------------------------------------------------
// kernels: reset, scan, statistics
// ---------------------------------------------------------------------------

// Mark every block free: free bitmap bits [0, n_l) set on every level, the
// other bitmaps and the object bitmaps zero (already cleared by memset).
__global__ void k_heap_mark_free(const __grid_constant__ dsr_dev_heap H, dsr_u64 M) {
    const dsr_u64 tid = (dsr_u64)blockIdx.x * blockDim.x + threadIdx.x;
    const dsr_u64 stride = (dsr_u64)gridDim.x * blockDim.x;
    const dsr_u64 f = 1ull << H.free_bm.shift;
    dsr_u64 n = M;
    for (int l = 0; l < H.free_bm.n_levels; ++l) {
        const dsr_u64 nw = H.free_bm.nwords[l];
        for (dsr_u64 i = tid; i < nw; i += stride) {
            const dsr_u64 lo = i * f;
            const dsr_u64 k = n - lo >= f ? f : n - lo;
            H.free_bm.lvl[l][i] = k >= 64 ? ~0ull : ((1ull << k) - 1);
        }
        n = (n + f - 1) / f;
    }
    for (dsr_u64 b = tid; b < M; b += stride) H.btype[b] = 0xFF;
}

// Do-all steps 1 and 2 (Section 2.3, Fig. 4): list the set bits of
// allocated[T] (step 1) and compact them into the block list R by a prefix
// sum (step 2). One thread per block id: each CTA takes 256 consecutive
// block ids per round; a warp ballots which of its 32 ids are allocated, the
// CTA forms the exclusive prefix sum of its 8 warp counts in shared memory
// and reserves its run of R with one atomicAdd; every listed block gets its
// id and the snapshot of its occupied slots. Runs of R follow block order
// within a round, so consecutive entries are usually neighbouring blocks.
// `types` is a bit mask: a do-all over a type with subtypes lists the blocks
// of every type in its subtree, one type after the other.
__global__ void __launch_bounds__(256) k_scan(const __grid_constant__ dsr_dev_heap H, uint32_t types,
                                              unsigned visits_mult) {
    __shared__ unsigned warp_n[8];
    __shared__ unsigned run_base;
    const dsr_u64 M = H.M;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned objs = 0;
    for (uint32_t tm = types; tm; tm &= tm - 1) {
        const int T = __ffs(tm) - 1;
        const dsr_u64* leaf = H.alloc_bm[T].lvl[0];
        const unsigned fsh = H.alloc_bm[T].shift, flo = (1u << fsh) - 1;
        const dsr_u64 v = H.valid[T];
        for (dsr_u64 base = (dsr_u64)blockIdx.x * 256; base < M; base += (dsr_u64)gridDim.x * 256) {
            const dsr_u64 b = base + threadIdx.x;
            const bool set = b < M && ((leaf[b >> fsh] >> (b & flo)) & 1ull);
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
                run_base = total ? atomicAdd(H.R_count, total) : 0;
            }
            __syncthreads();
            if (set) {
                const dsr_u64 live = v & ~H.obj[b];
                const unsigned k = run_base + warp_n[warp] + __popc(ballot & ((1u << lane) - 1));
                H.R_bid[k] = (uint32_t)b;
                H.R_mask[k] = live;
                objs += __popcll(live);
            }
            __syncthreads();
        }
    }
    objs = __reduce_add_sync(0xFFFFFFFFu, objs);
    if (lane == 0 && objs) dsr_count(H.ctr, DSR_CTR_VISITS, (dsr_u64)objs * visits_mult);
}

// Statistics: out[0] free blocks; out[1 + 3T + {0,1,2}] allocated blocks,
// active blocks, live objects of type T. Bit b of leaf word i stands for
// block (i << shift) + b, shift = log2 of the bitmap fan-out (64, 32 or 16).
__global__ void k_stats(const __grid_constant__ dsr_dev_heap H, dsr_u64* out) {
    const dsr_u64 tid = (dsr_u64)blockIdx.x * blockDim.x + threadIdx.x;
    const dsr_u64 stride = (dsr_u64)gridDim.x * blockDim.x;
    const dsr_u64 nw = H.free_bm.nwords[0];
    dsr_u64 nfree = 0;
    for (dsr_u64 i = tid; i < nw; i += stride) nfree += __popcll(H.free_bm.lvl[0][i]);
    if (nfree) atomicAdd(out, nfree);
    for (int t = 0; t < H.n_types; ++t) {
        dsr_u64 na = 0, nact = 0, live = 0;
        const dsr_u64 v = H.valid[t];
        const unsigned sh = H.alloc_bm[t].shift;
        for (dsr_u64 i = tid; i < nw; i += stride) {
            dsr_u64 a = H.alloc_bm[t].lvl[0][i];
            na += __popcll(a);
            nact += __popcll(H.active_bm[t].lvl[0][i]);
            while (a) {
                const int b = __ffsll((long long)a) - 1;
                a &= a - 1;
                live += __popcll(v & ~H.obj[(i << sh) + (dsr_u64)b]);
            }
        }
        if (na) atomicAdd(out + 1 + 3 * t, na);
        if (nact) atomicAdd(out + 2 + 3 * t, nact);
        if (live) atomicAdd(out + 3 + 3 * t, live);
    }
}

bool dsr__vec4_ok(const dsr_heap* h, int type) {
    const dsr_layout& L = h->layout;
    if (h->dev.sub[type] != (1u << type)) return false;  // run4 takes one type
    if (L.capacity[type] % 4 || L.block_bytes % 16) return false;
    for (uint32_t f = 0; f < L.n_fields[type]; ++f)
        if (L.field_offset[type][f] % 16 || L.field_bytes[type][f] != 4) return false;
    return true;
}

int dsr__scan_grid(const dsr_heap* h, int type) {
    (void)type;
    uint64_t ctas = (h->dev.M + 255) / 256;
    const uint64_t cap = (uint64_t)h->sm_count * 8;
    if (ctas > cap) ctas = cap;
    return ctas < 1 ? 1 : (int)ctas;
}

void dsr__launch_scan(const dsr_heap* h, int type, cudaStream_t s, unsigned visits_per_object, bool exact) {
    const uint32_t types = exact ? (1u << type) : h->dev.sub[type];
    k_scan<<<dsr__scan_grid(h, type), 256, 0, s>>>(h->dev, types, visits_per_object);
}

int dsr__persistent_grid(const dsr_heap* h, const void* kernel, int threads) {
    int per_sm = h->tune.ctas_per_sm;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
    }
    return per_sm * h->sm_count;
}

// ---------------------------------------------------------------------------
// create / destroy / reset / layout
// ---------------------------------------------------------------------------
static void build_dev_view(dsr_heap* h) {
    const dsr_layout& L = h->layout;
    dsr_dev_heap& D = h->dev;
    memset(&D, 0, sizeof D);
    uint8_t* a = h->arena;
    D.data = a + L.off_data;
    D.obj = reinterpret_cast<dsr_u64*>(a + L.off_obj);
    D.btype = a + L.off_type;
    D.err = reinterpret_cast<uint32_t*>(a + DSR_HDR_ERR);
    D.inject = reinterpret_cast<uint32_t*>(a + DSR_HDR_INJECT);
    D.R_count = reinterpret_cast<uint32_t*>(a + DSR_HDR_RCOUNT);
    D.R_done = reinterpret_cast<uint32_t*>(a + DSR_HDR_RDONE);
    D.ctr = reinterpret_cast<dsr_u64*>(a + DSR_HDR_CTR);
    D.slow = reinterpret_cast<uint32_t*>(a + DSR_HDR_SLOW);
    // At most four block initialisations in flight per SM per type, and no
    // more than one per 64 blocks of the heap, so that a small heap is not
    // carved into nearly empty blocks by a burst of concurrent leaders.
    uint64_t sm = 4 * (uint64_t)(h->sm_count > 0 ? h->sm_count : 1), by_size = L.n_blocks / 64;
    D.slow_max = (uint32_t)(by_size < 1 ? 1 : (by_size < sm ? by_size : sm));
    D.dbg = reinterpret_cast<dsr_u64*>(a + DSR_HDR_DBG);
    D.R_mask = reinterpret_cast<dsr_u64*>(a + off_rmask(L));
    D.R_bid = reinterpret_cast<uint32_t*>(a + off_rbid(L));
    D.M = L.n_blocks;
    D.block_bytes = L.block_bytes;
    D.n_types = (int32_t)L.n_types;
    auto fill = [&](dsr_hbm& b, uint64_t off) {
        b.n_levels = (int32_t)L.n_levels;
        b.shift = L.fanout == 16 ? 4u : L.fanout == 32 ? 5u : 6u;
        uint64_t o = off;
        for (uint32_t l = 0; l < L.n_levels; ++l) {
            b.lvl[l] = reinterpret_cast<dsr_u64*>(a + o);
            b.nwords[l] = (uint32_t)L.words_per_level[l];
            o += L.words_per_level[l] * 8;
        }
    };
    fill(D.free_bm, L.off_free_bm);
    for (uint32_t t = 0; t < L.n_types; ++t) {
        fill(D.alloc_bm[t], L.off_alloc_bm + t * L.bitmap_words * 8);
        fill(D.active_bm[t], L.off_active_bm + t * L.bitmap_words * 8);
        D.cap[t] = L.capacity[t];
        D.valid[t] = L.capacity[t] >= 64 ? ~0ull : ((1ull << L.capacity[t]) - 1);
        D.n_fields[t] = L.n_fields[t];
        for (uint32_t f = 0; f < L.n_fields[t]; ++f) {
            D.foff[t][f] = L.field_offset[t][f];
            D.fsize[t][f] = (uint8_t)L.field_bytes[t][f];
        }
        D.sub[t] = 1u << t;  // no subtypes until dsr_heap_set_bases
        D.span_sh[t] = L.capacity[t] <= 32 ? 5 : 6;
    }
    h->stats_dev = reinterpret_cast<dsr_u64*>(a + DSR_HDR_STATS);
}

static int reset_impl(dsr_heap* h, cudaStream_t s) {
    const dsr_layout& L = h->layout;
    cudaError_t e;
    e = cudaMemsetAsync(h->arena, 0, DSR_HEADER_BYTES, s);
    if (!e) e = cudaMemsetAsync(h->arena + L.off_free_bm, 0, (1 + 2 * L.n_types) * L.bitmap_words * 8, s);
    if (!e) e = cudaMemsetAsync(h->arena + L.off_obj, 0, L.n_blocks * 8, s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_heap_reset");
        return DSR_E_CUDA;
    }
    uint64_t ctas = (L.n_blocks + 255) / 256;
    if (ctas > (uint64_t)h->sm_count * 16) ctas = (uint64_t)h->sm_count * 16;
    if (ctas < 1) ctas = 1;
    k_heap_mark_free<<<(unsigned)ctas, 256, 0, s>>>(h->dev, L.n_blocks);
    return dsr__check_launch("k_heap_mark_free");
}

extern "C" int dsr_heap_create(const dsr_type_desc* types, int n_types, void* arena_dev, size_t heap_bytes,
                               const dsr_tuning* tune, void* stream, dsr_heap** out) {
    if (!out || !arena_dev || (reinterpret_cast<uintptr_t>(arena_dev) & 255)) return DSR_E_INVALID;
    *out = nullptr;
    dsr_tuning tn = resolve_tuning(tune);
    if (tn.threads < 64 || tn.threads > 1024 || tn.threads % 64) return DSR_E_INVALID;
    dsr_layout L;
    int rc = geometry(types, n_types, tn, &L);
    if (rc) return rc;
    // Largest M that fits: estimate, then step down.
    const uint64_t per_block = L.block_bytes + 8 + 8 + 4 + 1 + (1 + 2 * (uint64_t)n_types) * 2;
    if (heap_bytes < DSR_HEADER_BYTES + 4096 + per_block) return DSR_E_OOM;
    uint64_t M = (heap_bytes - DSR_HEADER_BYTES - 4096) / per_block;
    if (M > 0xFFFFFFFFull) M = 0xFFFFFFFFull;
    while (M > 0 && place(&L, M) > heap_bytes) M -= 1 + M / 4096;
    if (M == 0) return DSR_E_OOM;
    while (place(&L, M + 1) <= heap_bytes && M < 0xFFFFFFFFull) ++M;
    place(&L, M);

    dsr_heap* h = new (std::nothrow) dsr_heap;
    if (!h) return DSR_E_OOM;
    h->layout = L;
    h->arena = static_cast<uint8_t*>(arena_dev);
    h->heap_bytes = heap_bytes;
    h->tune = tn;
    cudaError_t e = cudaGetDevice(&h->device);
    if (!e) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    if (e) {
        dsr__set_cuda_error(e, "dsr_heap_create");
        delete h;
        return DSR_E_CUDA;
    }
    build_dev_view(h);
    rc = reset_impl(h, dsr__stream(stream));
    if (rc) {
        delete h;
        return rc;
    }
    *out = h;
    return DSR_OK;
}

// ---------------------------------------------------------------------------
// subtypes (Section 1: class inheritance without wasted memory)
// ---------------------------------------------------------------------------
// Validates base[] against the types' fields and writes each type's subtree
// mask: bit u of sub[t] is set iff u is t or a (transitive) subtype of t.
static int type_tree(int n_types, const uint32_t* n_fields, const uint32_t (*field_bytes)[DSR_MAX_FIELDS],
                     const int* base, uint32_t* sub) {
    if (n_types < 1 || n_types > DSR_MAX_TYPES || !base || !sub) return DSR_E_INVALID;
    for (int t = 0; t < n_types; ++t) {
        const int b = base[t];
        if (b < -1 || b >= t) return DSR_E_INVALID;  // a base is declared before its subtypes
        if (b < 0) continue;
        // the inherited fields come first, with the base's sizes, so a field
        // index means the same field in the base and in every subtype
        if (n_fields[t] < n_fields[b]) return DSR_E_INVALID;
        for (uint32_t f = 0; f < n_fields[b]; ++f)
            if (field_bytes[t][f] != field_bytes[b][f]) return DSR_E_INVALID;
    }
    for (int t = 0; t < n_types; ++t) sub[t] = 1u << t;
    for (int t = n_types - 1; t >= 0; --t)  // subtypes have higher indices: children before parents
        if (base[t] >= 0) sub[base[t]] |= sub[t];
    return DSR_OK;
}

extern "C" int dsr_type_tree(const dsr_type_desc* types, int n_types, const int* base, uint32_t* sub_out) {
    if (!types || n_types < 1 || n_types > DSR_MAX_TYPES) return DSR_E_INVALID;
    uint32_t nf[DSR_MAX_TYPES];
    uint32_t fb[DSR_MAX_TYPES][DSR_MAX_FIELDS];
    for (int t = 0; t < n_types; ++t) {
        if (types[t].n_fields < 1 || types[t].n_fields > DSR_MAX_FIELDS || !types[t].field_bytes)
            return DSR_E_INVALID;
        nf[t] = (uint32_t)types[t].n_fields;
        for (int f = 0; f < types[t].n_fields; ++f) fb[t][f] = (uint32_t)types[t].field_bytes[f];
    }
    return type_tree(n_types, nf, fb, base, sub_out);
}

extern "C" int dsr_heap_set_bases(dsr_heap* h, const int* base) {
    if (!h) return DSR_E_INVALID;
    const dsr_layout& L = h->layout;
    uint32_t sub[DSR_MAX_TYPES];
    const int rc = type_tree((int)L.n_types, L.n_fields, L.field_bytes, base, sub);
    if (rc) return rc;
    for (uint32_t t = 0; t < L.n_types; ++t) {
        h->dev.sub[t] = sub[t];
        uint8_t sh = 5;  // 64 threads per listed block if any visited type has more than 32 slots
        for (uint32_t u = 0; u < L.n_types; ++u)
            if (((sub[t] >> u) & 1u) && L.capacity[u] > 32) sh = 6;
        h->dev.span_sh[t] = sh;
    }
    h->version += 1;
    return DSR_OK;
}

extern "C" int dsr_heap_destroy(dsr_heap* h) {
    delete h;
    return DSR_OK;
}

extern "C" int dsr_heap_reset(dsr_heap* h, void* stream) {
    if (!h) return DSR_E_INVALID;
    return reset_impl(h, dsr__stream(stream));
}

extern "C" int dsr_heap_layout(const dsr_heap* h, dsr_layout* out) {
    if (!h || !out) return DSR_E_INVALID;
    *out = h->layout;
    return DSR_OK;
}

extern "C" size_t dsr_dev_heap_size(void) { return sizeof(dsr_dev_heap); }

extern "C" int dsr_heap_device_view(const dsr_heap* h, void* out, size_t out_bytes) {
    if (!h || !out || out_bytes < sizeof(dsr_dev_heap)) return DSR_E_INVALID;
    memcpy(out, &h->dev, sizeof(dsr_dev_heap));
    return DSR_OK;
}

extern "C" int dsr_heap_stats(dsr_heap* h, void* stream, dsr_stats* out) {
    if (!h || !out) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    const int n = 1 + 3 * DSR_MAX_TYPES;
    cudaError_t e = cudaMemsetAsync(h->stats_dev, 0, n * sizeof(dsr_u64), s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_heap_stats");
        return DSR_E_CUDA;
    }
    uint64_t ctas = (h->layout.words_per_level[0] + 255) / 256;
    if (ctas > (uint64_t)h->sm_count * 8) ctas = (uint64_t)h->sm_count * 8;
    if (ctas < 1) ctas = 1;
    k_stats<<<(unsigned)ctas, 256, 0, s>>>(h->dev, h->stats_dev);
    int rc = dsr__check_launch("k_stats");
    if (rc) return rc;
    dsr_u64 buf[1 + 3 * DSR_MAX_TYPES];
    uint32_t err = 0;
    e = cudaMemcpyAsync(buf, h->stats_dev, sizeof buf, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(&err, h->dev.err, sizeof err, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_heap_stats");
        return DSR_E_CUDA;
    }
    memset(out, 0, sizeof *out);
    out->n_blocks = h->layout.n_blocks;
    out->free_blocks = buf[0];
    out->n_types = h->layout.n_types;
    out->error_flags = err;
    for (uint32_t t = 0; t < h->layout.n_types; ++t) {
        out->capacity[t] = h->layout.capacity[t];
        out->allocated_blocks[t] = buf[1 + 3 * t];
        out->active_blocks[t] = buf[2 + 3 * t];
        out->live_objects[t] = buf[3 + 3 * t];
    }
    return DSR_OK;
}

extern "C" int dsr_heap_counters(dsr_heap* h, void* stream, uint64_t* out) {
    if (!h || !out) return DSR_E_INVALID;
    dsr_u64 rows[DSR_CTR_SLOTS][DSR_CTR_COUNT];
    cudaError_t e = cudaMemcpyAsync(rows, h->dev.ctr, sizeof rows, cudaMemcpyDeviceToHost, dsr__stream(stream));
    if (!e) e = cudaStreamSynchronize(dsr__stream(stream));
    if (e) {
        dsr__set_cuda_error(e, "dsr_heap_counters");
        return DSR_E_CUDA;
    }
    for (unsigned k = 0; k < DSR_CTR_COUNT; ++k) {
        out[k] = 0;
        for (unsigned r = 0; r < DSR_CTR_SLOTS; ++r) out[k] += rows[r][k];
    }
    return DSR_OK;
}

extern "C" int dsr_heap_check_record(dsr_heap* h, uint32_t* err_out, uint64_t* record_out) {
    if (!h) return DSR_E_INVALID;
    uint32_t e32 = 0;
    dsr_u64 rec = 0;
    cudaError_t e = cudaMemcpy(&e32, h->dev.err, 4, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(&rec, h->dev.dbg, 8, cudaMemcpyDeviceToHost);
    if (e) {
        dsr__set_cuda_error(e, "dsr_heap_check_record");
        return DSR_E_CUDA;
    }
    if (err_out) *err_out = e32;
    if (record_out) *record_out = rec;
    return DSR_OK;
}

extern "C" int dsr_heap_inject_oom(dsr_heap* h, uint32_t n, void* stream) {
    if (!h) return DSR_E_INVALID;
    cudaError_t e = cudaMemcpyAsync(h->dev.inject, &n, sizeof n, cudaMemcpyHostToDevice, dsr__stream(stream));
    if (!e) e = cudaStreamSynchronize(dsr__stream(stream));  // n lives on this stack frame
    if (e) {
        dsr__set_cuda_error(e, "dsr_heap_inject_oom");
        return DSR_E_CUDA;
    }
    return DSR_OK;
}

// ---------------------------------------------------------------------------
// generic methods
// ---------------------------------------------------------------------------
struct MCount {
    typedef dsr_count_args Args;
    static __device__ void run(const dsr_dev_heap&, int, const Args& a, dsr_ref) {
        // one atomic per warp
        const unsigned act = __activemask();
        if (dsr_lane() == (unsigned)(__ffs(act) - 1)) atomicAdd(a.counter_dev, (dsr_u64)__popc(act));
    }
};

// field f += field f + 1 for every field but the last, which gets + 1.
struct MStreamAdd {
    struct Args { int dummy; };
    static __device__ void run(const dsr_dev_heap& H, int T, const Args&, dsr_ref r) {
        const int nf = (int)H.n_fields[T];
        for (int f = 0; f + 1 < nf; ++f) {
            int32_t* p = dsr_field<int32_t>(H, T, r, f);
            *p += *dsr_field<int32_t>(H, T, r, f + 1);
        }
        *dsr_field<int32_t>(H, T, r, nf - 1) += 1;
    }
    // Four slots at once: all NF field vectors are loaded before any store,
    // so a thread has NF 16-byte loads in flight.
    template <int NF>
    static __device__ __forceinline__ void quad(const dsr_dev_heap& H, int T, uint32_t bid, unsigned s0, unsigned live) {
        uint8_t* base = H.data + (dsr_u64)bid * H.block_bytes + 4 * s0;
        int4 v[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) v[f] = *reinterpret_cast<const int4*>(base + H.foff[T][f]);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            int4 o = v[f];
            if (f + 1 < NF) {
                o.x += v[f + 1].x, o.y += v[f + 1].y, o.z += v[f + 1].z, o.w += v[f + 1].w;
            } else {
                o.x += 1, o.y += 1, o.z += 1, o.w += 1;
            }
            int32_t* p = reinterpret_cast<int32_t*>(base + H.foff[T][f]);
            if (live == 0xFu) {
                *reinterpret_cast<int4*>(p) = o;
            } else {
                if (live & 1u) p[0] = o.x;
                if (live & 2u) p[1] = o.y;
                if (live & 4u) p[2] = o.z;
                if (live & 8u) p[3] = o.w;
            }
        }
    }
    static __device__ void run4(const dsr_dev_heap& H, int T, const Args&, uint32_t bid, unsigned s0, unsigned live) {
        switch (H.n_fields[T]) {
            case 1: quad<1>(H, T, bid, s0, live); break;
            case 2: quad<2>(H, T, bid, s0, live); break;
            case 3: quad<3>(H, T, bid, s0, live); break;
            case 4: quad<4>(H, T, bid, s0, live); break;
            case 5: quad<5>(H, T, bid, s0, live); break;
            case 6: quad<6>(H, T, bid, s0, live); break;
            case 7: quad<7>(H, T, bid, s0, live); break;
            case 8: quad<8>(H, T, bid, s0, live); break;
            default:  // wider types: one slot at a time
                for (unsigned k = 0; k < 4; ++k)
                    if (live & (1u << k)) run(H, T, Args{0}, ((dsr_u64)bid << 6) | (s0 + k));
        }
    }
};

struct MDeleteIf {
    typedef dsr_delete_if_args Args;
    static __device__ void run(const dsr_dev_heap& H, int T, const Args& a, dsr_ref r) {
        const int32_t v = *dsr_field<int32_t>(H, T, r, 0);
        int32_t m = v % a.modulus;
        if (m < 0) m += a.modulus;
        if (m == a.residue) dsr_delete(H, r);
    }
};

struct MClone {
    typedef dsr_clone_args Args;
    static __device__ void run(const dsr_dev_heap& H, int T, const Args& a, dsr_ref r) {
        const dsr_ref n = dsr_new(H, a.dst_type);
        if (n == DSR_NULL) return;
        const int nf = (int)(H.n_fields[T] < H.n_fields[a.dst_type] ? H.n_fields[T] : H.n_fields[a.dst_type]);
        for (int f = 0; f < nf; ++f) *dsr_field<int32_t>(H, a.dst_type, n, f) = *dsr_field<int32_t>(H, T, r, f) + a.add;
        for (int f = nf; f < (int)H.n_fields[a.dst_type]; ++f) *dsr_field<int32_t>(H, a.dst_type, n, f) = 0;
    }
};

struct DumpArgs {
    uint32_t* out;
    dsr_u64* count;
    dsr_u64 cap;
    int row;
};
struct MDump {
    typedef DumpArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int T, const Args& a, dsr_ref r) {
        const dsr_u64 k = atomicAdd(a.count, 1ull);
        if (k >= a.cap) {
            atomicOr(H.err, DSR_ERR_CAPACITY);
            return;
        }
        uint32_t* row = a.out + k * (dsr_u64)a.row;
        int w = 0;
        for (uint32_t f = 0; f < H.n_fields[T]; ++f) {
            if (H.fsize[T][f] == 4) {
                row[w++] = *dsr_field<uint32_t>(H, T, r, (int)f);
            } else {
                const dsr_u64 x = *dsr_field<dsr_u64>(H, T, r, (int)f);
                row[w++] = (uint32_t)x;
                row[w++] = (uint32_t)(x >> 32);
            }
        }
        row[w++] = (uint32_t)r;
        row[w++] = (uint32_t)(r >> 32);
    }
};

struct HashArgs {
    dsr_u64* out;
};
struct MHash {
    typedef HashArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int T, const Args& a, dsr_ref r) {
        dsr_u64 h = dsr_mix64((dsr_u64)T + DSR_GAMMA);
        for (uint32_t f = 0; f < H.n_fields[T]; ++f) {
            if (H.fsize[T][f] == 4) {
                h = dsr_mix64((h ^ (dsr_u64)*dsr_field<uint32_t>(H, T, r, (int)f)) + DSR_GAMMA);
            } else {
                const dsr_u64 x = *dsr_field<dsr_u64>(H, T, r, (int)f);
                h = dsr_mix64((h ^ (dsr_u64)(uint32_t)x) + DSR_GAMMA);
                h = dsr_mix64((h ^ (x >> 32)) + DSR_GAMMA);
            }
        }
        // Warp sum modulo 2^64 in three 22-bit chunks (each chunk sum of 32
        // lanes fits 32 bits), one atomic per warp.
        const unsigned act = __activemask();
        const dsr_u64 s0 = __reduce_add_sync(act, (unsigned)(h & 0x3FFFFFu));
        const dsr_u64 s1 = __reduce_add_sync(act, (unsigned)((h >> 22) & 0x3FFFFFu));
        const dsr_u64 s2 = __reduce_add_sync(act, (unsigned)(h >> 44));
        h = s0 + (s1 << 22) + (s2 << 44);
        if (dsr_lane() == (unsigned)(__ffs(act) - 1)) atomicAdd(a.out, h);
    }
};

extern "C" int dsr_row_words(const dsr_heap* h, int type) {
    if (!h || type < 0 || type >= (int)h->layout.n_types) return -1;
    int w = 2;
    for (uint32_t f = 0; f < h->layout.n_fields[type]; ++f) w += (int)h->layout.field_bytes[type][f] / 4;
    return w;
}

extern "C" int dsr_heap_dump(dsr_heap* h, int type, void* out_dev, uint64_t cap, void* count_dev, void* stream) {
    if (!h || !out_dev || !count_dev || type < 0 || type >= (int)h->layout.n_types) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    cudaError_t e = cudaMemsetAsync(count_dev, 0, sizeof(dsr_u64), s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_heap_dump");
        return DSR_E_CUDA;
    }
    DumpArgs a{static_cast<uint32_t*>(out_dev), static_cast<dsr_u64*>(count_dev), cap, dsr_row_words(h, type)};
    return dsr__doall<MDump>(h, type, a, s, true, nullptr, nullptr, 0, true);
}

extern "C" int dsr_heap_hash(dsr_heap* h, int type, void* hash_dev, void* stream) {
    if (!h || !hash_dev || type < 0 || type >= (int)h->layout.n_types) return DSR_E_INVALID;
    HashArgs a{static_cast<dsr_u64*>(hash_dev)};
    return dsr__doall<MHash>(h, type, a, dsr__stream(stream), true, nullptr, nullptr, 0, true);
}

template <class M>
static int typed_args(const void* args, size_t bytes, typename M::Args* out) {
    if (bytes != sizeof(typename M::Args) || !args) return DSR_E_INVALID;
    memcpy(out, args, sizeof *out);
    return DSR_OK;
}

// True if every field of every type in the mask is 4 bytes wide.
static bool all_fields_4(const dsr_layout& L, uint32_t types) {
    for (uint32_t t = 0; t < L.n_types; ++t)
        if ((types >> t) & 1u)
            for (uint32_t f = 0; f < L.n_fields[t]; ++f)
                if (L.field_bytes[t][f] != 4) return false;
    return true;
}

static int dispatch(dsr_heap* h, int type, int method, const void* args, size_t args_bytes, cudaStream_t s,
                    bool with_scan) {
    if (!h || type < 0 || type >= (int)h->layout.n_types) return DSR_E_INVALID;
    const uint32_t visited = h->dev.sub[type];  // type and its subtypes
    switch (method) {
        case DSR_METHOD_COUNT: {
            MCount::Args a;
            if (typed_args<MCount>(args, args_bytes, &a) || !a.counter_dev) return DSR_E_INVALID;
            return dsr__doall<MCount>(h, type, a, s, with_scan);
        }
        case DSR_METHOD_STREAM_ADD: {
            if (!all_fields_4(h->layout, visited)) return DSR_E_INVALID;
            return dsr__doall<MStreamAdd>(h, type, MStreamAdd::Args{0}, s, with_scan);
        }
        case DSR_METHOD_DELETE_IF: {
            MDeleteIf::Args a;
            if (typed_args<MDeleteIf>(args, args_bytes, &a) || a.modulus <= 0) return DSR_E_INVALID;
            if (h->layout.field_bytes[type][0] != 4) return DSR_E_INVALID;
            return dsr__doall<MDeleteIf>(h, type, a, s, with_scan);
        }
        case DSR_METHOD_CLONE: {
            MClone::Args a;
            if (typed_args<MClone>(args, args_bytes, &a)) return DSR_E_INVALID;
            // the clones are not visited: dst_type must lie outside the visited subtree
            if (a.dst_type < 0 || a.dst_type >= (int)h->layout.n_types || ((visited >> a.dst_type) & 1u))
                return DSR_E_INVALID;
            if (!all_fields_4(h->layout, visited | (1u << a.dst_type))) return DSR_E_INVALID;
            return dsr__doall<MClone>(h, type, a, s, with_scan);
        }
        default:
            break;
    }
    if (method >= 100 && method < 200) return dsr__gol_method(h, type, method, args, args_bytes, s, with_scan);
    if (method >= 200 && method < 300) return dsr__wator_method(h, type, method, args, args_bytes, s, with_scan);
    if (method >= 300 && method < 400) return dsr__nbody_method(h, type, method, args, args_bytes, s, with_scan);
    return DSR_E_INVALID;
}

extern "C" int dsr_parallel_do(dsr_heap* h, int type, int method, const void* args, size_t args_bytes,
                               void* stream) {
    return dispatch(h, type, method, args, args_bytes, dsr__stream(stream), true);
}

extern "C" int dsr_doall_scan(dsr_heap* h, int type, void* stream) {
    if (!h || type < 0 || type >= (int)h->layout.n_types) return DSR_E_INVALID;
    dsr__launch_scan(h, type, dsr__stream(stream));
    return dsr__check_launch("k_scan");
}

extern "C" int dsr_doall_run(dsr_heap* h, int type, int method, const void* args, size_t args_bytes, void* stream) {
    return dispatch(h, type, method, args, args_bytes, dsr__stream(stream), false);
}

// ---------------------------------------------------------------------------
// allocation microbenchmark kernels
// ---------------------------------------------------------------------------
// The microbenchmark loops run warp-uniform trip counts (the bound is
// rounded up to whole warps) and reconverge the warp at every iteration, so
// that each dsr_new / dsr_delete call sees the whole warp.
__global__ void k_bench_alloc(const __grid_constant__ dsr_dev_heap H, dsr_u64 n, int n_types, dsr_u64 seed,
                              dsr_ref* refs) {
    const dsr_u64 stride = (dsr_u64)gridDim.x * blockDim.x;
    const dsr_u64 n32 = (n + 31) & ~31ull;
    for (dsr_u64 i = (dsr_u64)blockIdx.x * blockDim.x + threadIdx.x; i < n32; i += stride) {
        __syncwarp();
        if (i >= n) continue;
        const int T = (int)(dsr_mix64(seed ^ (i * DSR_GAMMA)) % (dsr_u64)n_types);
        const dsr_ref r = dsr_new(H, T);
        if (r != DSR_NULL) *dsr_field<int32_t>(H, T, r, 0) = (int32_t)i;
        refs[i] = r;
    }
}

__global__ void k_bench_free(const __grid_constant__ dsr_dev_heap H, dsr_u64 n, const dsr_ref* refs) {
    const dsr_u64 stride = (dsr_u64)gridDim.x * blockDim.x;
    const dsr_u64 n32 = (n + 31) & ~31ull;
    for (dsr_u64 i = (dsr_u64)blockIdx.x * blockDim.x + threadIdx.x; i < n32; i += stride) {
        __syncwarp();
        if (i < n) dsr_delete(H, refs[i]);
    }
}

__global__ void k_bench_churn(const __grid_constant__ dsr_dev_heap H, dsr_u64 n, int n_types, dsr_u64 seed,
                              dsr_ref* refs, unsigned long long* n_replaced) {
    const dsr_u64 stride = (dsr_u64)gridDim.x * blockDim.x;
    const dsr_u64 n32 = (n + 31) & ~31ull;
    unsigned long long mine = 0;
    for (dsr_u64 i = (dsr_u64)blockIdx.x * blockDim.x + threadIdx.x; i < n32; i += stride) {
        __syncwarp();
        if (i >= n || !(dsr_mix64(seed ^ (i * DSR_GAMMA)) & 1)) continue;
        dsr_delete(H, refs[i]);
        const int T = (int)(dsr_mix64((seed + 1) ^ (i * DSR_GAMMA)) % (dsr_u64)n_types);
        const dsr_ref r = dsr_new(H, T);
        if (r != DSR_NULL) *dsr_field<int32_t>(H, T, r, 0) = (int32_t)i;
        refs[i] = r;
        ++mine;
    }
    // one atomic per warp
    for (int o = 16; o; o >>= 1) mine += __shfl_down_sync(0xFFFFFFFFu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(n_replaced, mine);
}

// 8 independent chains per thread keep the FMA pipes busy; the result is
// written so that nothing is eliminated.
__global__ void k_bench_fma(float* out, int iters) {
    const float b = 0.999999f, c = 1e-7f;
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
    }
    float sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

extern "C" int dsr_bench_churn(dsr_heap* h, uint64_t n, int n_types_used, uint64_t seed, void* refs_dev,
                               void* n_replaced_dev, void* stream) {
    if (!h || !refs_dev || !n_replaced_dev || n_types_used < 1 || n_types_used > (int)h->layout.n_types || n == 0)
        return DSR_E_INVALID;
    for (int t = 0; t < n_types_used; ++t)
        if (h->layout.field_bytes[t][0] != 4) return DSR_E_INVALID;
    uint64_t ctas = (n + 255) / 256;
    if (ctas > (uint64_t)h->sm_count * 8) ctas = (uint64_t)h->sm_count * 8;
    k_bench_churn<<<(unsigned)ctas, 256, 0, dsr__stream(stream)>>>(
        h->dev, n, n_types_used, seed, static_cast<dsr_ref*>(refs_dev), static_cast<unsigned long long*>(n_replaced_dev));
    return dsr__check_launch("k_bench_churn");
}

// One word per thread: reductions (results unused) or dependent atomics.
__global__ void k_bench_atomics(dsr_u64* words, dsr_u64 n, int iters, int with_return) {
    const dsr_u64 i = (dsr_u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dsr_u64* w = words + i;
    const dsr_u64 bit = 1ull << (i & 63);
    if (with_return) {
        dsr_u64 acc = 0;
        for (int k = 0; k < iters; ++k) acc += (k & 1) ? atomicAnd(w, ~(bit ^ (acc & 1))) : atomicOr(w, bit | (acc & 2));
        if (acc == 0x5DEECE66Dull) *w = acc;  // keeps the results live
    } else {
        for (int k = 0; k < iters; ++k) {
            if (k & 1)
                atomicAnd(w, ~bit);
            else
                atomicOr(w, bit);
        }
    }
}

extern "C" int dsr_bench_atomics(void* words_dev, uint64_t n_words, int iters, int with_return, void* stream) {
    if (!words_dev || n_words == 0 || iters < 1) return DSR_E_INVALID;
    const dsr_u64 ctas = (n_words + 255) / 256;
    if (ctas > 0x7FFFFFFFull) return DSR_E_INVALID;
    k_bench_atomics<<<(unsigned)ctas, 256, 0, dsr__stream(stream)>>>(static_cast<dsr_u64*>(words_dev), n_words, iters,
                                                                     with_return);
    return dsr__check_launch("k_bench_atomics");
}

extern "C" int dsr_bench_fma(float* out_dev, int ctas, int iters, void* stream) {
    if (!out_dev || ctas < 1 || iters < 1) return DSR_E_INVALID;
    k_bench_fma<<<ctas, 256, 0, dsr__stream(stream)>>>(out_dev, iters);
    return dsr__check_launch("k_bench_fma");
}

extern "C" int dsr_bench_alloc(dsr_heap* h, uint64_t n, int n_types_used, uint64_t seed, void* refs_dev,
                               void* stream) {
    if (!h || !refs_dev || n_types_used < 1 || n_types_used > (int)h->layout.n_types || n == 0) return DSR_E_INVALID;
    for (int t = 0; t < n_types_used; ++t)
        if (h->layout.field_bytes[t][0] != 4) return DSR_E_INVALID;
    uint64_t ctas = (n + 255) / 256;
    if (ctas > (uint64_t)h->sm_count * 8) ctas = (uint64_t)h->sm_count * 8;
    k_bench_alloc<<<(unsigned)ctas, 256, 0, dsr__stream(stream)>>>(h->dev, n, n_types_used, seed,
                                                                      static_cast<dsr_ref*>(refs_dev));
    return dsr__check_launch("k_bench_alloc");
}

extern "C" int dsr_bench_free(dsr_heap* h, uint64_t n, const void* refs_dev, void* stream) {
    if (!h || !refs_dev || n == 0) return DSR_E_INVALID;
    uint64_t ctas = (n + 255) / 256;
    if (ctas > (uint64_t)h->sm_count * 8) ctas = (uint64_t)h->sm_count * 8;
    k_bench_free<<<(unsigned)ctas, 256, 0, dsr__stream(stream)>>>(h->dev, n, static_cast<const dsr_ref*>(refs_dev));
    return dsr__check_launch("k_bench_free");
}
