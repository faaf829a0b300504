// Traffic as an SMMO program (Fig. 6g, the Nagel-Schreckenberg model): R
// single-lane roads of L cells; Car objects move by the model's four rules in
// one do-all per step, Source objects (open roads) admit new cars in a second.
//
// Rules (parallel update; occupancy read at the start of the step):
//   do-all Car:    v1 = min(v + 1, vmax); g = free cells ahead, looking at
//                  most v1 cells ahead (open road: cells past the end are
//                  free; periodic road: wraps); v2 = min(v1, g); with
//                  probability p (draw rand(seed, 5, t, road * L + x))
//                  v3 = max(v2 - 1, 0), else v2; x' = x + v3; an open-road
//                  car with x' >= L leaves (delete this).
//   do-all Source: if cell 0 is free after the cars moved and the draw
//                  rand(seed, 6, t, road) is below alpha, new Car(road, 0,
//                  v_entry); otherwise count an entry blocked by a car.
// Occupancy lives in two byte grids: a step reads `cur` and marks the new
// positions in `next`, which must start empty. A car only moves into free
// cells ahead of it, before the next car, so no two cars mark one cell and
// no car reads a cell another car writes: the do-all needs no atomics. After
// the step `cur` is cleared and the grids swap.
#include "dsr_apps.h"
#include "dsr_internal.cuh"

namespace {
enum { CAR = 0, SOURCE = 1 };
enum { F_ROAD = 0, F_X = 1, F_V = 2 };             // Car
enum { S_ROAD = 0, S_ENTERED = 1, S_BLOCKED = 2 };  // Source
enum { CTR_ENTERED = DSR_CTR_APP0, CTR_LEFT, CTR_MOVED, CTR_VSUM };

struct TrafficArgs {
    const uint8_t* cur;  // [R * L] occupancy at the start of the step
    uint8_t* next;       // [R * L] occupancy after the step (zero on entry)
    dsr_traffic_params p;
    dsr_u64 step;
};

__device__ __forceinline__ int32_t* fld(const dsr_dev_heap& H, int T, dsr_ref r, int f) {
    return dsr_field<int32_t>(H, T, r, f);
}

__device__ __forceinline__ bool draws_below(dsr_u64 r, dsr_u64 thr) { return (r >> 32) < thr; }

struct MCar {
    typedef TrafficArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        const int32_t road = *fld(H, CAR, self, F_ROAD), x = *fld(H, CAR, self, F_X), v = *fld(H, CAR, self, F_V);
        const int32_t L = a.p.L;
        const uint8_t* row = a.cur + (dsr_u64)road * L;
        const int32_t v1 = v + 1 < a.p.vmax ? v + 1 : a.p.vmax;
        int32_t g = 0;
        for (; g < v1; ++g) {
            int32_t ahead = x + g + 1;
            if (ahead >= L) {
                if (!a.p.periodic) continue;  // past the end of an open road: free
                ahead -= L;
            }
            if (row[ahead]) break;
        }
        int32_t v3 = v1 < g ? v1 : g;
        if (draws_below(dsr_rand(a.p.seed, 5, a.step, (dsr_u64)road * L + x), a.p.p_thr)) v3 = v3 > 0 ? v3 - 1 : 0;
        // flow statistics: one atomic per warp for each
        const unsigned act = __activemask();
        const unsigned vsum = __reduce_add_sync(act, (unsigned)v3);
        const unsigned moved = __popc(__ballot_sync(act, v3 > 0));
        if (dsr_lane() == (unsigned)(__ffs(act) - 1)) {
            if (moved) dsr_count(H.ctr, CTR_MOVED, moved);
            if (vsum) dsr_count(H.ctr, CTR_VSUM, vsum);
        }
        int32_t nx = x + v3;
        if (nx >= L) {
            if (!a.p.periodic) {
                dsr_count_lanes(H.ctr, CTR_LEFT);
                dsr_delete(H, self);
                return;
            }
            nx -= L;
        }
        a.next[(dsr_u64)road * L + nx] = 1;
        *fld(H, CAR, self, F_X) = nx;
        *fld(H, CAR, self, F_V) = v3;
    }
};

struct MSource {
    typedef TrafficArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        const int32_t road = *fld(H, SOURCE, self, S_ROAD);
        uint8_t* cell0 = a.next + (dsr_u64)road * a.p.L;
        if (*cell0) {
            *fld(H, SOURCE, self, S_BLOCKED) += 1;
            return;
        }
        if (!draws_below(dsr_rand(a.p.seed, 6, a.step, (dsr_u64)road), a.p.a_thr)) return;
        const dsr_ref c = dsr_new(H, CAR);
        if (c == DSR_NULL) return;  // out of memory: DSR_ERR_OOM is set
        *fld(H, CAR, c, F_ROAD) = road;
        *fld(H, CAR, c, F_X) = 0;
        *fld(H, CAR, c, F_V) = a.p.v_entry;
        *cell0 = 1;
        *fld(H, SOURCE, self, S_ENTERED) += 1;
        dsr_count_lanes(H.ctr, CTR_ENTERED);
    }
};

// One thread per cell: a Car where v0 >= 0, and on open roads a Source per
// road (made by the thread of cell 0).
__global__ void k_traffic_init(const __grid_constant__ dsr_dev_heap H, const int8_t* v0, uint8_t* cur,
                               dsr_traffic_params p) {
    const dsr_u64 n = (dsr_u64)p.R * p.L;
    const dsr_u64 n32 = (n + 31) & ~31ull;  // warp-uniform trip count
    for (dsr_u64 i = (dsr_u64)blockIdx.x * blockDim.x + threadIdx.x; i < n32; i += (dsr_u64)gridDim.x * blockDim.x) {
        __syncwarp();  // whole-warp groups for dsr_new
        if (i >= n) continue;
        const int32_t road = (int32_t)(i / p.L), x = (int32_t)(i % p.L);
        const int v = v0[i];
        if (v >= 0) {
            const dsr_ref c = dsr_new(H, CAR);
            if (c != DSR_NULL) {
                *fld(H, CAR, c, F_ROAD) = road;
                *fld(H, CAR, c, F_X) = x;
                *fld(H, CAR, c, F_V) = v < p.vmax ? v : p.vmax;
                cur[i] = 1;
            }
        }
        if (!p.periodic && x == 0) {
            const dsr_ref s = dsr_new(H, SOURCE);
            if (s != DSR_NULL) {
                *fld(H, SOURCE, s, S_ROAD) = road;
                *fld(H, SOURCE, s, S_ENTERED) = 0;
                *fld(H, SOURCE, s, S_BLOCKED) = 0;
            }
        }
    }
}

const int kCarFields[3] = {4, 4, 4};
const int kSourceFields[3] = {4, 4, 4};

bool heap_matches(const dsr_heap* h) {
    const dsr_layout& L = h->layout;
    if (L.n_types < 2 || L.n_fields[CAR] != 3 || L.n_fields[SOURCE] != 3) return false;
    for (int t = 0; t < 2; ++t)
        for (int f = 0; f < 3; ++f)
            if (L.field_bytes[t][f] != 4) return false;
    return true;
}

bool params_ok(const dsr_traffic_params* p) {
    return p && p->R >= 1 && p->vmax >= 1 && p->vmax <= 127 && p->L > p->vmax && p->v_entry >= 0 &&
           p->v_entry <= p->vmax && (int64_t)p->R * p->L <= (1ll << 40) && p->p_thr <= (1ull << 32) &&
           p->a_thr <= (1ull << 32);
}

size_t grid_bytes(const dsr_traffic_params& p) { return ((size_t)p.R * p.L + 255) / 256 * 256; }
}  // namespace

struct dsr_traffic {
    dsr_heap* heap;
    dsr_traffic_params p;
    uint8_t* grid[2];
    int cur;         // index of the grid holding the current occupancy
    dsr_u64 step;    // steps taken
};

extern "C" int dsr_traffic_types(dsr_type_desc* out) {
    if (!out) return DSR_E_INVALID;
    out[0] = dsr_type_desc{"Car", 3, kCarFields};
    out[1] = dsr_type_desc{"Source", 3, kSourceFields};
    return DSR_OK;
}

extern "C" int dsr_traffic_workspace_bytes(const dsr_traffic_params* p, size_t* out) {
    if (!out || !params_ok(p)) return DSR_E_INVALID;
    *out = 2 * grid_bytes(*p);
    return DSR_OK;
}

extern "C" int dsr_traffic_create(dsr_heap* heap, const dsr_traffic_params* p, const void* v0_dev,
                                  void* workspace_dev, void* stream, dsr_traffic** out) {
    if (!heap || !v0_dev || !workspace_dev || !out || !params_ok(p) || !heap_matches(heap)) return DSR_E_INVALID;
    if (reinterpret_cast<uintptr_t>(workspace_dev) & 255) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    dsr_traffic* t = new dsr_traffic;
    t->heap = heap;
    t->p = *p;
    t->grid[0] = static_cast<uint8_t*>(workspace_dev);
    t->grid[1] = t->grid[0] + grid_bytes(*p);
    t->cur = 0;
    t->step = 0;
    cudaError_t e = cudaMemsetAsync(workspace_dev, 0, 2 * grid_bytes(*p), s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_traffic_create");
        delete t;
        return DSR_E_CUDA;
    }
    const dsr_u64 n = (dsr_u64)p->R * p->L;
    dsr_u64 ctas = (n + 255) / 256;
    if (ctas > (dsr_u64)heap->sm_count * 8) ctas = (dsr_u64)heap->sm_count * 8;
    k_traffic_init<<<(unsigned)ctas, 256, 0, s>>>(heap->dev, static_cast<const int8_t*>(v0_dev), t->grid[0], *p);
    int rc = dsr__check_launch("k_traffic_init");
    if (rc) {
        delete t;
        return rc;
    }
    *out = t;
    return DSR_OK;
}

extern "C" int dsr_traffic_step(dsr_traffic* t, int n_steps, void* stream) {
    if (!t || n_steps < 0) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    for (int i = 0; i < n_steps; ++i) {
        TrafficArgs a{t->grid[t->cur], t->grid[1 - t->cur], t->p, t->step};
        int rc = dsr__doall<MCar>(t->heap, CAR, a, s);
        if (!rc && !t->p.periodic) rc = dsr__doall<MSource>(t->heap, SOURCE, a, s);
        if (rc) return rc;
        cudaError_t e = cudaMemsetAsync(t->grid[t->cur], 0, grid_bytes(t->p), s);  // the next step's `next`
        if (e) {
            dsr__set_cuda_error(e, "dsr_traffic_step");
            return DSR_E_CUDA;
        }
        t->cur = 1 - t->cur;
        t->step += 1;
    }
    return DSR_OK;
}

extern "C" int dsr_traffic_occupancy(const dsr_traffic* t, const void** grid_dev) {
    if (!t || !grid_dev) return DSR_E_INVALID;
    *grid_dev = t->grid[t->cur];
    return DSR_OK;
}

extern "C" int dsr_traffic_destroy(dsr_traffic* t) {
    delete t;
    return DSR_OK;
}
