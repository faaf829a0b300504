// BitmapAlloc comparator: host API, the do-all scan, statistics and the
// state hash (see dsr_bitmap_alloc.cuh).
#include <new>
#include <vector>

#include "dsr_apps.h"
#include "dsr_bitmap_alloc.cuh"

// Arena: header (err, R counters, check record, event counters, as a dsr heap
// header) | per type: bitmap words, object array | R word ids | R masks.
static const size_t kBmHeader = DSR_HEADER_BYTES;

static inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

static int bm_geometry(const dsr_type_desc* types, int n_types, const uint64_t* cap, uint32_t obj_bytes[],
                       uint16_t foff[][DSR_MAX_FIELDS], uint32_t n_fields[], uint32_t fbytes[][DSR_MAX_FIELDS],
                       size_t* total) {
    if (!types || !cap || n_types < 1 || n_types > DSR_MAX_TYPES) return DSR_E_INVALID;
    size_t off = kBmHeader, max_words = 0;
    for (int t = 0; t < n_types; ++t) {
        const dsr_type_desc& d = types[t];
        if (d.n_fields < 1 || d.n_fields > DSR_MAX_FIELDS || !d.field_bytes) return DSR_E_INVALID;
        if (cap[t] == 0 || cap[t] % 64 || cap[t] > (64ull << 31)) return DSR_E_INVALID;
        uint32_t o = 0, align = 4;
        for (int f = 0; f < d.n_fields; ++f) {
            const int b = d.field_bytes[f];
            if (b != 4 && b != 8) return DSR_E_INVALID;
            o = (o + (uint32_t)b - 1) / (uint32_t)b * (uint32_t)b;
            if (foff) foff[t][f] = (uint16_t)o;
            if (fbytes) fbytes[t][f] = (uint32_t)b;
            o += (uint32_t)b;
            if ((uint32_t)b > align) align = (uint32_t)b;
        }
        o = (o + align - 1) / align * align;
        if (obj_bytes) obj_bytes[t] = o;
        if (n_fields) n_fields[t] = (uint32_t)d.n_fields;
        off += up256(cap[t] / 8);      // bitmap
        off += up256(cap[t] * o);      // objects
        if (cap[t] / 64 > max_words) max_words = cap[t] / 64;
    }
    off += up256(max_words * 4) + up256(max_words * 8);
    *total = off;
    return DSR_OK;
}

extern "C" int dsr_bm_heap_bytes(const dsr_type_desc* types, int n_types, const uint64_t* capacity, size_t* out) {
    if (!out) return DSR_E_INVALID;
    return bm_geometry(types, n_types, capacity, nullptr, nullptr, nullptr, nullptr, out);
}

extern "C" int dsr_bm_heap_create(const dsr_type_desc* types, int n_types, const uint64_t* capacity, void* arena_dev,
                                  size_t arena_bytes, void* stream, dsr_bm_heap** out) {
    if (!out || !arena_dev || (reinterpret_cast<uintptr_t>(arena_dev) & 255)) return DSR_E_INVALID;
    *out = nullptr;
    dsr_bm_heap* h = new (std::nothrow) dsr_bm_heap;
    if (!h) return DSR_E_OOM;
    memset(h, 0, sizeof *h);
    size_t need = 0;
    int rc = bm_geometry(types, n_types, capacity, h->dev.obj_bytes, h->dev.foff, h->n_fields, h->field_bytes, &need);
    if (rc || need > arena_bytes) {
        delete h;
        return rc ? rc : DSR_E_OOM;
    }
    uint8_t* a = static_cast<uint8_t*>(arena_dev);
    h->arena = a;
    h->n_types = n_types;
    h->dev.n_types = n_types;
    h->dev.err = reinterpret_cast<uint32_t*>(a + DSR_HDR_ERR);
    h->dev.R_count = reinterpret_cast<uint32_t*>(a + DSR_HDR_RCOUNT);
    h->dev.R_done = reinterpret_cast<uint32_t*>(a + DSR_HDR_RDONE);
    h->dev.dbg = reinterpret_cast<dsr_u64*>(a + DSR_HDR_DBG);
    h->dev.ctr = reinterpret_cast<dsr_u64*>(a + DSR_HDR_CTR);
    size_t off = kBmHeader, max_words = 0;
    for (int t = 0; t < n_types; ++t) {
        h->dev.cap[t] = capacity[t];
        h->dev.used[t] = reinterpret_cast<dsr_u64*>(a + off);
        off += up256(capacity[t] / 8);
        h->dev.data[t] = a + off;
        off += up256(capacity[t] * h->dev.obj_bytes[t]);
        if (capacity[t] / 64 > max_words) max_words = capacity[t] / 64;
    }
    h->dev.R_word = reinterpret_cast<uint32_t*>(a + off);
    off += up256(max_words * 4);
    h->dev.R_mask = reinterpret_cast<dsr_u64*>(a + off);
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || h->sm_count < 1)
        h->sm_count = 1;
    // every slot free: zero the header and the bitmaps
    cudaStream_t s = dsr__stream(stream);
    cudaError_t e = cudaMemsetAsync(a, 0, kBmHeader, s);
    for (int t = 0; t < n_types && !e; ++t) e = cudaMemsetAsync(h->dev.used[t], 0, capacity[t] / 8, s);
    if (e) {
        delete h;
        dsr__set_cuda_error(e, "dsr_bm_heap_create");
        return DSR_E_CUDA;
    }
    *out = h;
    return DSR_OK;
}

extern "C" int dsr_bm_heap_destroy(dsr_bm_heap* h) {
    delete h;
    return DSR_OK;
}

// List the non-zero bitmap words of type T into R (CTA-level compaction, one
// atomicAdd per 256 words); count the listed objects `mult` times as visits.
__global__ void __launch_bounds__(256) k_bm_scan(const __grid_constant__ dsr_bm_dev H, int T, unsigned mult) {
    __shared__ unsigned warp_n[8];
    __shared__ unsigned run_base;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const dsr_u64 nw = H.cap[T] >> 6;
    unsigned objs = 0;
    for (dsr_u64 base = (dsr_u64)blockIdx.x * 256; base < nw; base += (dsr_u64)gridDim.x * 256) {
        const dsr_u64 i = base + threadIdx.x;
        const dsr_u64 w = i < nw ? H.used[T][i] : 0;
        const unsigned ballot = __ballot_sync(0xFFFFFFFFu, w != 0);
        if (lane == 0) warp_n[warp] = __popc(ballot);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned total = 0;
            for (int k = 0; k < 8; ++k) {
                const unsigned n = warp_n[k];
                warp_n[k] = total;
                total += n;
            }
            run_base = total ? atomicAdd(H.R_count, total) : 0;
        }
        __syncthreads();
        if (w) {
            const unsigned k = run_base + warp_n[warp] + __popc(ballot & ((1u << lane) - 1));
            H.R_word[k] = (uint32_t)i;
            H.R_mask[k] = w;
            objs += __popcll(w);
        }
        __syncthreads();
    }
    objs = __reduce_add_sync(0xFFFFFFFFu, objs);
    if (lane == 0 && objs) dsr_count(H.ctr, DSR_CTR_VISITS, (dsr_u64)objs * mult);
}

void dsr__bm_launch_scan(const dsr_bm_heap* h, int type, cudaStream_t s, unsigned visits_per_object) {
    const dsr_u64 nw = h->dev.cap[type] >> 6;
    dsr_u64 ctas = (nw + 255) / 256;
    if (ctas > (dsr_u64)h->sm_count * 8) ctas = (dsr_u64)h->sm_count * 8;
    if (ctas < 1) ctas = 1;
    k_bm_scan<<<(unsigned)ctas, 256, 0, s>>>(h->dev, type, visits_per_object);
}

int dsr__bm_grid(const dsr_bm_heap* h, const void* kernel, int threads) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * h->sm_count;
}

namespace {
struct BmHashArgs {
    dsr_u64* out;
};
// The object-state hash of dsr_heap_hash, over the 32-bit field words.
struct BmHash {
    typedef BmHashArgs Args;
    static __device__ void run(const dsr_bm_dev& H, int T, const Args& a, dsr_ref r) {
        dsr_u64 h = dsr_mix64((dsr_u64)T + DSR_GAMMA);
        const uint32_t* w = dsr_field<uint32_t>(H, T, r, 0);
        for (uint32_t k = 0; k < H.obj_bytes[T] / 4; ++k) h = dsr_mix64((h ^ (dsr_u64)w[k]) + DSR_GAMMA);
        const unsigned act = __activemask();
        const dsr_u64 s0 = __reduce_add_sync(act, (unsigned)(h & 0x3FFFFFu));
        const dsr_u64 s1 = __reduce_add_sync(act, (unsigned)((h >> 22) & 0x3FFFFFu));
        const dsr_u64 s2 = __reduce_add_sync(act, (unsigned)(h >> 44));
        h = s0 + (s1 << 22) + (s2 << 44);
        if (dsr_lane() == (unsigned)(__ffs(act) - 1)) atomicAdd(a.out, h);
    }
};

__global__ void k_bm_count(const __grid_constant__ dsr_bm_dev H, int T, dsr_u64* out) {
    const dsr_u64 nw = H.cap[T] >> 6;
    unsigned long long n = 0;
    for (dsr_u64 i = (dsr_u64)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += (dsr_u64)gridDim.x * blockDim.x)
        n += __popcll(H.used[T][i]);
    for (int o = 16; o; o >>= 1) n += __shfl_down_sync(0xFFFFFFFFu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(reinterpret_cast<unsigned long long*>(out), n);
}
}  // namespace

extern "C" int dsr_bm_heap_hash(dsr_bm_heap* h, int type, void* hash_dev, void* stream) {
    if (!h || !hash_dev || type < 0 || type >= h->n_types) return DSR_E_INVALID;
    for (uint32_t f = 0; f < h->n_fields[type]; ++f)
        if (h->field_bytes[type][f] != 4) return DSR_E_INVALID;  // the hash reads 32-bit fields
    return dsr__bm_doall<BmHash>(h, type, BmHashArgs{static_cast<dsr_u64*>(hash_dev)}, dsr__stream(stream));
}

extern "C" int dsr_bm_heap_stats(dsr_bm_heap* h, void* stream, uint64_t* live_out, uint32_t* err_out) {
    if (!h || !live_out) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    dsr_u64* scratch = reinterpret_cast<dsr_u64*>(h->arena + DSR_HDR_STATS);
    cudaError_t e = cudaMemsetAsync(scratch, 0, 8 * DSR_MAX_TYPES, s);
    for (int t = 0; t < h->n_types && !e; ++t) {
        k_bm_count<<<h->sm_count * 4, 256, 0, s>>>(h->dev, t, scratch + t);
        e = cudaGetLastError();
    }
    uint32_t err = 0;
    if (!e) e = cudaMemcpyAsync(live_out, scratch, 8 * (size_t)h->n_types, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(&err, h->dev.err, 4, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_bm_heap_stats");
        return DSR_E_CUDA;
    }
    if (err_out) *err_out = err;
    return DSR_OK;
}

extern "C" int dsr_bm_heap_counters(dsr_bm_heap* h, void* stream, uint64_t* out) {
    if (!h || !out) return DSR_E_INVALID;
    std::vector<dsr_u64> rows((size_t)DSR_CTR_SLOTS * DSR_CTR_COUNT);
    cudaStream_t s = dsr__stream(stream);
    cudaError_t e = cudaMemcpyAsync(rows.data(), h->dev.ctr, rows.size() * 8, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_bm_heap_counters");
        return DSR_E_CUDA;
    }
    for (unsigned k = 0; k < DSR_CTR_COUNT; ++k) {
        out[k] = 0;
        for (unsigned r = 0; r < DSR_CTR_SLOTS; ++r) out[k] += rows[(size_t)r * DSR_CTR_COUNT + k];
    }
    return DSR_OK;
}
