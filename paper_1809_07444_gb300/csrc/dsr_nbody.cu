// N-body with merging collisions as an SMMO program (Fig. 6b "collisions"
// and 6d "nbody"; Fig. 1 names an Euler time step). FP32 on the device.
//
// One step is a do-all over Body whose block list R is built once and shared
// by four kernels (no body is created or deleted until the last one):
//   gather   each listed slot writes its body's position and mass to dense
//            arrays indexed by g = R index * 64 + slot (empty slots: mass 0);
//   force    a_i = G sum_j m_j d_ij / (|d_ij|^2 + eps^2)^(3/2) over all dense
//            entries, tiled through shared memory; then v += a dt, x += v dt
//            (semi-implicit Euler), written to the object and to a second
//            dense buffer;
//   partner  on the updated positions, the partner of i is the body with the
//            lowest id j != i within r_merge;
//   merge    mutual partners merge: the lower id takes the summed mass and
//            the mass-weighted position and velocity, the higher id deletes
//            itself.
// The last kernel's last CTA resets R.
#include <cfloat>
#include "dsr_apps.h"
#include "dsr_internal.cuh"

#include <mutex>

namespace {
enum { BODY = 0 };
enum { ID = 0, PX = 1, PY = 2, PZ = 3, VX = 4, VY = 5, VZ = 6, MASS = 7 };
constexpr int TILE = 256;

struct NbWs {
    float4* pos;      // [S] x, y, z, m before the update (m = 0: empty slot)
    float4* npos;     // [S] x, y, z, m after the update
    float4* nvel;     // [S] vx, vy, vz after the update
    int32_t* id;      // [S] body id, INT_MAX for an empty slot
    int32_t* partner; // [S] dense index of the partner, -1 if none
    float4* part;     // [ns][nt * TILE] acceleration sums per slice of j tiles (nullptr: unsplit kernels)
    int2* pbest;      // [ns][nt * TILE] lowest partner id and its index per slice
    int32_t* log;     // [log_cap][3] merges: step, survivor id, absorbed id
    dsr_u64* log_n;   // merges logged so far
    dsr_u64* step;    // device step counter
    dsr_u64 log_cap;
};

struct NbArgs {
    NbWs ws;
    dsr_nbody_params p;
};

__device__ __forceinline__ float* fld(const dsr_dev_heap& H, dsr_ref r, int f) { return dsr_field<float>(H, BODY, r, f); }

__device__ __forceinline__ float4 ws_load(const float4* p, uint32_t g, uint32_t n) {
    return g < n ? p[g] : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Compensated (Kahan) accumulation: s += x with the lost low part kept in c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Dense slot count of the current block list.
__device__ __forceinline__ uint32_t n_dense(const dsr_dev_heap& H) { return (*(volatile uint32_t*)H.R_count) << 6; }

__global__ void k_gather(const __grid_constant__ dsr_dev_heap H, NbWs ws) {
    const uint32_t n = n_dense(H);
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const uint32_t i = g >> 6, s = g & 63;
        if ((H.R_mask[i] >> s) & 1ull) {
            const dsr_ref r = ((dsr_u64)H.R_bid[i] << 6) | s;
            ws.pos[g] = make_float4(*fld(H, r, PX), *fld(H, r, PY), *fld(H, r, PZ), *fld(H, r, MASS));
            ws.id[g] = *dsr_field<int32_t>(H, BODY, r, ID);
        } else {
            ws.pos[g] = make_float4(0.f, 0.f, 0.f, 0.f);
            ws.id[g] = 0x7FFFFFFF;
        }
    }
}

// All-pairs force and the Euler update. One thread per dense slot; CTAs are
// uniform over the dense range, so a CTA either works or exits as a whole.
// Within a tile the 256 terms are summed in order; tile sums are added with
// Kahan compensation, so the accumulated rounding stays near one tile's.
__global__ void __launch_bounds__(TILE) k_force(const __grid_constant__ dsr_dev_heap H, NbArgs a) {
    __shared__ float4 sp[TILE];
    const uint32_t n = n_dense(H);
    const uint32_t base = blockIdx.x * TILE;
    if (base >= n) return;
    const uint32_t g = base + threadIdx.x;
    const float4 pi = ws_load(a.ws.pos, g, n);
    const float eps2 = a.p.eps * a.p.eps;
    float ax = 0.f, ay = 0.f, az = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    for (uint32_t t0 = 0; t0 < n; t0 += TILE) {
        __syncthreads();
        sp[threadIdx.x] = t0 + threadIdx.x < n ? a.ws.pos[t0 + threadIdx.x] : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        float tx = 0.f, ty = 0.f, tz = 0.f;
#pragma unroll 8
        for (int j = 0; j < TILE; ++j) {
            const float4 pj = sp[j];
            const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
            const float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
            const float w = pj.w * inv * inv * inv;
            tx = fmaf(w, dx, tx);
            ty = fmaf(w, dy, ty);
            tz = fmaf(w, dz, tz);
        }
        kahan_add(ax, cx, tx);
        kahan_add(ay, cy, ty);
        kahan_add(az, cz, tz);
    }
    if (g >= n) return;
    const uint32_t i = g >> 6, s = g & 63;
    if (!((H.R_mask[i] >> s) & 1ull)) {
        a.ws.npos[g] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const dsr_ref r = ((dsr_u64)H.R_bid[i] << 6) | s;
    const float G = a.p.G, dt = a.p.dt;
    const float vx = fmaf(G * ax, dt, *fld(H, r, VX));
    const float vy = fmaf(G * ay, dt, *fld(H, r, VY));
    const float vz = fmaf(G * az, dt, *fld(H, r, VZ));
    const float x = fmaf(vx, dt, pi.x), y = fmaf(vy, dt, pi.y), z = fmaf(vz, dt, pi.z);
    *fld(H, r, VX) = vx;
    *fld(H, r, VY) = vy;
    *fld(H, r, VZ) = vz;
    *fld(H, r, PX) = x;
    *fld(H, r, PY) = y;
    *fld(H, r, PZ) = z;
    a.ws.npos[g] = make_float4(x, y, z, pi.w);
    a.ws.nvel[g] = make_float4(vx, vy, vz, 0.f);
}

// Split form of the two all-pairs kernels, the one dsr_nbody_step runs.
//
// Work items. The unsplit kernels give one CTA per 256 bodies, under two CTAs
// per SM at 65,536 bodies. Here a row item is TILE * RB bodies (RB per
// thread), the j tiles are cut into `ns` slices, and a work item is one
// (row item, slice) pair; `ns` follows from the dense count on the device
// (n_slices), so the items fill about `grid` CTAs whatever the live count.
// Each item writes its partial result to part[slice][g] (pbest for the
// partner search); the combine kernels read the slices back in slice order,
// so the result does not depend on which CTA ran which item.
//
// Register blocking. Every lane of a warp reads the same j body from shared
// memory (a broadcast), and at one body per thread the shared-memory return
// path, not the FP32 pipe, sets the pace. With RB bodies per thread each
// load feeds RB pairs. A pair costs the same operations, rounded in the same
// order, as in k_force.
constexpr int RB = 4;  // bodies per thread in the split kernels

__device__ __forceinline__ uint32_t n_slices(uint32_t nr, uint32_t nj, uint32_t grid) {
    if (!nr) return 0;
    const uint32_t k = grid / nr;
    return k < 1 ? 1 : (k > nj ? nj : k);
}

struct SplitShape {
    uint32_t n, nj, nr, ns;  // dense count, j tiles, row items, slices
};

__device__ __forceinline__ SplitShape split_shape(const dsr_dev_heap& H, uint32_t grid) {
    SplitShape q;
    q.n = n_dense(H);
    q.nj = (q.n + TILE - 1) / TILE;
    q.nr = (q.n + TILE * RB - 1) / (TILE * RB);
    q.ns = n_slices(q.nr, q.nj, grid);
    return q;
}

// 1/sqrt(x) by the PTX approximate reciprocal square root with subnormal
// inputs flushed to zero; used only where x >= eps^2 >= FLT_MIN, so the
// flush never applies.
__device__ __forceinline__ float rsqrt_normal(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Acceleration sums of one slice of j tiles for RB bodies per thread (body k
// of a thread: row * TILE * RB + k * TILE + threadIdx.x), compensated across
// tiles as in k_force. SOFT: eps^2 >= FLT_MIN, so r^2 >= eps^2 is a normal
// number for every pair, the body itself included, and neither the
// zero-distance guard nor subnormal handling is needed.
template <bool SOFT>
__global__ void __launch_bounds__(TILE) k_force_part(const __grid_constant__ dsr_dev_heap H, NbArgs a) {
    __shared__ float4 sp[TILE];
    const SplitShape q = split_shape(H, gridDim.x);
    const float eps2 = a.p.eps * a.p.eps;
    for (uint32_t item = blockIdx.x; item < q.nr * q.ns; item += gridDim.x) {
        const uint32_t row = item % q.nr, sl = item / q.nr;
        const uint32_t g0 = row * TILE * RB + threadIdx.x;
        float px[RB], py[RB], pz[RB];
        float ax[RB], ay[RB], az[RB], cx[RB], cy[RB], cz[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            const float4 u = ws_load(a.ws.pos, g0 + k * TILE, q.n);
            px[k] = u.x, py[k] = u.y, pz[k] = u.z;
            ax[k] = ay[k] = az[k] = cx[k] = cy[k] = cz[k] = 0.f;
        }
        for (uint32_t t = q.nj * sl / q.ns; t < q.nj * (sl + 1) / q.ns; ++t) {
            __syncthreads();
            sp[threadIdx.x] = ws_load(a.ws.pos, t * TILE + threadIdx.x, q.n);
            __syncthreads();
            float tx[RB], ty[RB], tz[RB];
#pragma unroll
            for (int k = 0; k < RB; ++k) tx[k] = ty[k] = tz[k] = 0.f;
#pragma unroll 4
            for (int j = 0; j < TILE; ++j) {
                const float4 pj = sp[j];
#pragma unroll
                for (int k = 0; k < RB; ++k) {
                    const float dx = pj.x - px[k], dy = pj.y - py[k], dz = pj.z - pz[k];
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                    const float inv = SOFT ? rsqrt_normal(r2) : (r2 > 0.f ? rsqrtf(r2) : 0.f);
                    const float w = pj.w * inv * inv * inv;
                    tx[k] = fmaf(w, dx, tx[k]);
                    ty[k] = fmaf(w, dy, ty[k]);
                    tz[k] = fmaf(w, dz, tz[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                kahan_add(ax[k], cx[k], tx[k]);
                kahan_add(ay[k], cy[k], ty[k]);
                kahan_add(az[k], cz[k], tz[k]);
            }
        }
        float4* out = a.ws.part + (size_t)sl * q.nr * TILE * RB;
#pragma unroll
        for (int k = 0; k < RB; ++k)
            if (g0 + k * TILE < q.n) out[g0 + k * TILE] = make_float4(ax[k], ay[k], az[k], 0.f);
    }
}

// Slice sums (compensated, in slice order) -> acceleration -> the Euler
// update of k_force. `grid` is k_force_part's grid.
__global__ void k_force_combine(const __grid_constant__ dsr_dev_heap H, NbArgs a, uint32_t grid) {
    const SplitShape q = split_shape(H, grid);
    const size_t stride = (size_t)q.nr * TILE * RB;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < q.n; g += gridDim.x * blockDim.x) {
        const uint32_t i = g >> 6, s = g & 63;
        if (!((H.R_mask[i] >> s) & 1ull)) {
            a.ws.npos[g] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        float ax = 0.f, ay = 0.f, az = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
        for (uint32_t k = 0; k < q.ns; ++k) {
            const float4 v = a.ws.part[k * stride + g];
            kahan_add(ax, cx, v.x);
            kahan_add(ay, cy, v.y);
            kahan_add(az, cz, v.z);
        }
        const float4 pi = a.ws.pos[g];
        const dsr_ref r = ((dsr_u64)H.R_bid[i] << 6) | s;
        const float G = a.p.G, dt = a.p.dt;
        const float vx = fmaf(G * ax, dt, *fld(H, r, VX));
        const float vy = fmaf(G * ay, dt, *fld(H, r, VY));
        const float vz = fmaf(G * az, dt, *fld(H, r, VZ));
        const float x = fmaf(vx, dt, pi.x), y = fmaf(vy, dt, pi.y), z = fmaf(vz, dt, pi.z);
        *fld(H, r, VX) = vx;
        *fld(H, r, VY) = vy;
        *fld(H, r, VZ) = vz;
        *fld(H, r, PX) = x;
        *fld(H, r, PY) = y;
        *fld(H, r, PZ) = z;
        a.ws.npos[g] = make_float4(x, y, z, pi.w);
        a.ws.nvel[g] = make_float4(vx, vy, vz, 0.f);
    }
}

// Partner search over one slice of j tiles for RB bodies per thread: per
// body the lowest partner id in the slice and that partner's dense index.
// The distance test fails for almost every pair, so the common path is the
// squared distances and one test of their minimum; the per-body
// tests, the mass and the id (read from the gathered ids) sit behind it. Ids
// are unique, so "not itself" is j != g.
__global__ void __launch_bounds__(TILE) k_partner_part(const __grid_constant__ dsr_dev_heap H, NbArgs a) {
    __shared__ float4 sp[TILE];
    const SplitShape q = split_shape(H, gridDim.x);
    const float rm2 = a.p.r_merge * a.p.r_merge;
    for (uint32_t item = blockIdx.x; item < q.nr * q.ns; item += gridDim.x) {
        const uint32_t row = item % q.nr, sl = item / q.nr;
        const uint32_t g0 = row * TILE * RB + threadIdx.x;
        float px[RB], py[RB], pz[RB];
        int32_t best_id[RB], best[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            const float4 u = ws_load(a.ws.npos, g0 + k * TILE, q.n);
            px[k] = u.x, py[k] = u.y, pz[k] = u.z;
            best_id[k] = 0x7FFFFFFF, best[k] = -1;
        }
        for (uint32_t t = q.nj * sl / q.ns; t < q.nj * (sl + 1) / q.ns; ++t) {
            const uint32_t t0 = t * TILE;
            __syncthreads();
            sp[threadIdx.x] = ws_load(a.ws.npos, t0 + threadIdx.x, q.n);
            __syncthreads();
#pragma unroll 4
            for (int j = 0; j < TILE; ++j) {
                const float4 pj = sp[j];
                float d2[RB];
#pragma unroll
                for (int k = 0; k < RB; ++k) {
                    const float dx = pj.x - px[k], dy = pj.y - py[k], dz = pj.z - pz[k];
                    d2[k] = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                }
                float dmin = d2[0];
#pragma unroll
                for (int k = 1; k < RB; ++k) dmin = fminf(dmin, d2[k]);
                if (dmin < rm2 && pj.w > 0.f) {
                    const uint32_t jg = t0 + j;
#pragma unroll
                    for (int k = 0; k < RB; ++k) {
                        if (d2[k] < rm2 && jg != g0 + k * TILE) {
                            const int32_t jid = a.ws.id[jg];
                            if (jid < best_id[k]) {
                                best_id[k] = jid;
                                best[k] = (int32_t)jg;
                            }
                        }
                    }
                }
            }
        }
        int2* out = a.ws.pbest + (size_t)sl * q.nr * TILE * RB;
#pragma unroll
        for (int k = 0; k < RB; ++k)
            if (g0 + k * TILE < q.n) out[g0 + k * TILE] = make_int2(best_id[k], best[k]);
    }
}

// The partner over all slices: the lowest id (ids are unique).
__global__ void k_partner_combine(const __grid_constant__ dsr_dev_heap H, NbArgs a, uint32_t grid) {
    const SplitShape q = split_shape(H, grid);
    const size_t stride = (size_t)q.nr * TILE * RB;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < q.n; g += gridDim.x * blockDim.x) {
        int2 b = make_int2(0x7FFFFFFF, -1);
        for (uint32_t k = 0; k < q.ns; ++k) {
            const int2 v = a.ws.pbest[k * stride + g];
            if (v.x < b.x) b = v;
        }
        a.ws.partner[g] = a.ws.npos[g].w > 0.f ? b.y : -1;
    }
}

// Partner search on the updated positions: lowest id within r_merge.
__global__ void __launch_bounds__(TILE) k_partner(const __grid_constant__ dsr_dev_heap H, NbArgs a) {
    __shared__ float4 sp[TILE];
    __shared__ int32_t sid[TILE];
    const uint32_t n = n_dense(H);
    const uint32_t base = blockIdx.x * TILE;
    if (base >= n) return;
    const uint32_t g = base + threadIdx.x;
    const float4 pi = g < n ? a.ws.npos[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int32_t myid = g < n ? a.ws.id[g] : 0x7FFFFFFF;
    const float rm2 = a.p.r_merge * a.p.r_merge;
    int32_t best_id = 0x7FFFFFFF, best = -1;
    for (uint32_t t0 = 0; t0 < n; t0 += TILE) {
        __syncthreads();
        const uint32_t j = t0 + threadIdx.x;
        sp[threadIdx.x] = j < n ? a.ws.npos[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        sid[threadIdx.x] = j < n ? a.ws.id[j] : 0x7FFFFFFF;
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < TILE; ++k) {
            const float4 pj = sp[k];
            const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const int32_t jid = sid[k];
            if (d2 < rm2 && jid < best_id && jid != myid && pj.w > 0.f) {
                best_id = jid;
                best = (int32_t)(t0 + k);
            }
        }
    }
    if (g < n) a.ws.partner[g] = (pi.w > 0.f) ? best : -1;
}

// Merge mutual partners; the higher id deletes itself. Last kernel of the
// step: its last CTA resets R and advances the step counter.
__global__ void k_merge(const __grid_constant__ dsr_dev_heap H, NbArgs a) {
    const uint32_t n = n_dense(H);
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t g = base + threadIdx.x;
        if (g >= n) continue;
        const int32_t j = a.ws.partner[g];
        if (j < 0 || a.ws.partner[j] != (int32_t)g) continue;
        const uint32_t i = g >> 6, s = g & 63;
        const dsr_ref r = ((dsr_u64)H.R_bid[i] << 6) | s;
        if (a.ws.id[g] > a.ws.id[j]) {
            dsr_delete(H, r);
            continue;
        }
        const float4 pg = a.ws.npos[g], pj = a.ws.npos[j];
        const float4 vg = a.ws.nvel[g], vj = a.ws.nvel[j];
        const float M = pg.w + pj.w;
        *fld(H, r, VX) = (pg.w * vg.x + pj.w * vj.x) / M;
        *fld(H, r, VY) = (pg.w * vg.y + pj.w * vj.y) / M;
        *fld(H, r, VZ) = (pg.w * vg.z + pj.w * vj.z) / M;
        *fld(H, r, PX) = (pg.w * pg.x + pj.w * pj.x) / M;
        *fld(H, r, PY) = (pg.w * pg.y + pj.w * pj.y) / M;
        *fld(H, r, PZ) = (pg.w * pg.z + pj.w * pj.z) / M;
        *fld(H, r, MASS) = M;
        const dsr_u64 k = atomicAdd(a.ws.log_n, 1ull);
        if (k < a.ws.log_cap) {
            a.ws.log[3 * k + 0] = (int32_t)*a.ws.step;
            a.ws.log[3 * k + 1] = a.ws.id[g];
            a.ws.log[3 * k + 2] = a.ws.id[j];
        }
    }
    if (dsr_doall_finish(H)) *a.ws.step += 1;
}

__global__ void k_nbody_init(const __grid_constant__ dsr_dev_heap H, const float* rows, int n) {
    const int n32 = (n + 31) & ~31;  // warp-uniform trip count
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n32; i += gridDim.x * blockDim.x) {
        __syncwarp();  // whole-warp groups for dsr_new
        if (i >= n) continue;
        const dsr_ref r = dsr_new(H, BODY);
        if (r == DSR_NULL) continue;
        *dsr_field<int32_t>(H, BODY, r, ID) = i;
        for (int f = 0; f < 7; ++f) *fld(H, r, PX + f) = rows[7 * i + f];
    }
}

const int kBodyFields[8] = {4, 4, 4, 4, 4, 4, 4, 4};

bool heap_matches(const dsr_heap* h) {
    const dsr_layout& L = h->layout;
    if (L.n_types < 1 || L.n_fields[BODY] != 8) return false;
    for (int f = 0; f < 8; ++f)
        if (L.field_bytes[BODY][f] != 4) return false;
    return true;
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Grid of a split all-pairs kernel: four waves of its resident CTAs.
uint32_t split_grid(const dsr_heap* h, const void* kernel) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, TILE, 0) != cudaSuccess || occ < 1) occ = 1;
    return (uint32_t)(4 * occ * h->sm_count);
}

struct SplitGrids {
    uint32_t force, partner;
};

SplitGrids split_grids(const dsr_heap* h) {
    return {split_grid(h, (const void*)k_force_part<true>), split_grid(h, (const void*)k_partner_part)};
}

// Slice entries: ns * nr <= max(grid, nr) items of TILE * RB bodies.
size_t split_slots(uint64_t S, SplitGrids g) {
    const uint64_t nr = (S + TILE * RB - 1) / (TILE * RB);
    uint64_t m = g.force > g.partner ? g.force : g.partner;
    if (nr > m) m = nr;
    return (size_t)m * TILE * RB;
}

size_t ws_bytes(uint64_t S, uint64_t log_cap, SplitGrids grid) {
    return 3 * round256(S * 16) + 2 * round256(S * 4) + round256(log_cap * 12) + 256 +
           round256(split_slots(S, grid) * 16) + round256(split_slots(S, grid) * 8);
}

NbWs carve(void* base, uint64_t S, uint64_t log_cap, SplitGrids grid) {
    uint8_t* p = static_cast<uint8_t*>(base);
    NbWs w;
    w.pos = reinterpret_cast<float4*>(p);
    p += round256(S * 16);
    w.npos = reinterpret_cast<float4*>(p);
    p += round256(S * 16);
    w.nvel = reinterpret_cast<float4*>(p);
    p += round256(S * 16);
    w.id = reinterpret_cast<int32_t*>(p);
    p += round256(S * 4);
    w.partner = reinterpret_cast<int32_t*>(p);
    p += round256(S * 4);
    w.log = reinterpret_cast<int32_t*>(p);
    p += round256(log_cap * 12);
    w.log_n = reinterpret_cast<dsr_u64*>(p);
    w.step = reinterpret_cast<dsr_u64*>(p + 8);
    p += 256;
    w.part = reinterpret_cast<float4*>(p);
    p += round256(split_slots(S, grid) * 16);
    w.pbest = reinterpret_cast<int2*>(p);
    w.log_cap = log_cap;
    return w;
}
}  // namespace

struct dsr_nbody {
    dsr_heap* heap;
    NbArgs args;
    uint64_t S;
    SplitGrids grid;  // of the split all-pairs kernels
};

extern "C" int dsr_nbody_types(dsr_type_desc* out) {
    if (!out) return DSR_E_INVALID;
    out[0] = dsr_type_desc{"Body", 8, kBodyFields};
    return DSR_OK;
}

extern "C" int dsr_nbody_workspace_bytes(const dsr_heap* heap, uint64_t log_cap, size_t* out) {
    if (!heap || !out) return DSR_E_INVALID;
    *out = ws_bytes(heap->layout.n_blocks * 64, log_cap, split_grids(heap));
    return DSR_OK;
}

extern "C" int dsr_nbody_create(dsr_heap* heap, const dsr_nbody_params* p, const void* rows_dev, int n_bodies,
                                void* workspace_dev, uint64_t log_cap, void* stream, dsr_nbody** out) {
    if (!heap || !p || !rows_dev || !workspace_dev || !out || n_bodies < 1) return DSR_E_INVALID;
    if ((reinterpret_cast<uintptr_t>(workspace_dev) & 255) || !heap_matches(heap)) return DSR_E_INVALID;
    if ((uint64_t)n_bodies > heap->layout.n_blocks * heap->layout.capacity[BODY]) return DSR_E_INVALID;
    dsr_nbody* nb = new dsr_nbody;
    nb->heap = heap;
    nb->S = heap->layout.n_blocks * 64;
    nb->grid = split_grids(heap);
    nb->args.ws = carve(workspace_dev, nb->S, log_cap, nb->grid);
    nb->args.p = *p;
    cudaStream_t s = dsr__stream(stream);
    cudaError_t e = cudaMemsetAsync(nb->args.ws.log_n, 0, 16, s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_nbody_create");
        delete nb;
        return DSR_E_CUDA;
    }
    int ctas = (n_bodies + 255) / 256;
    if (ctas > heap->sm_count * 8) ctas = heap->sm_count * 8;
    k_nbody_init<<<ctas, 256, 0, s>>>(heap->dev, static_cast<const float*>(rows_dev), n_bodies);
    int rc = dsr__check_launch("k_nbody_init");
    if (rc) {
        delete nb;
        return rc;
    }
    *out = nb;
    return DSR_OK;
}

extern "C" int dsr_nbody_step(dsr_nbody* nb, int n_steps, void* stream) {
    if (!nb || n_steps < 0) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    dsr_heap* h = nb->heap;
    const unsigned stream_ctas = (unsigned)(h->sm_count * 4);
    for (int i = 0; i < n_steps; ++i) {
        dsr__launch_scan(h, BODY, s);
        k_gather<<<stream_ctas, 256, 0, s>>>(h->dev, nb->args.ws);
        if (nb->args.p.eps * nb->args.p.eps >= FLT_MIN)
            k_force_part<true><<<nb->grid.force, TILE, 0, s>>>(h->dev, nb->args);
        else
            k_force_part<false><<<nb->grid.force, TILE, 0, s>>>(h->dev, nb->args);
        k_force_combine<<<stream_ctas, 256, 0, s>>>(h->dev, nb->args, nb->grid.force);
        k_partner_part<<<nb->grid.partner, TILE, 0, s>>>(h->dev, nb->args);
        k_partner_combine<<<stream_ctas, 256, 0, s>>>(h->dev, nb->args, nb->grid.partner);
        k_merge<<<stream_ctas, 256, 0, s>>>(h->dev, nb->args);
        int rc = dsr__check_launch("dsr_nbody_step");
        if (rc) return rc;
    }
    return DSR_OK;
}

extern "C" int dsr_nbody_merge_log(dsr_nbody* nb, void** log_dev, void** count_dev) {
    if (!nb || !log_dev || !count_dev) return DSR_E_INVALID;
    *log_dev = nb->args.ws.log;
    *count_dev = nb->args.ws.log_n;
    return DSR_OK;
}

extern "C" int dsr_nbody_destroy(dsr_nbody* nb) {
    delete nb;
    return DSR_OK;
}

int dsr__nbody_method(dsr_heap*, int, int, const void*, size_t, cudaStream_t, bool) { return DSR_E_INVALID; }

// ---------------------------------------------------------------------------
// Allocation-free step. The per-slot scratch of a step (dense positions,
// velocities, ids and partners) lives in this file-scope device array instead
// of a caller-allocated workspace, for callers that cannot call cudaMalloc.
// Every GPU that loads the library holds the array until the process exits.
// ---------------------------------------------------------------------------
namespace {
struct NoallocScratch {
    float4 pos[DSR_NOALLOC_MAX_SLOTS];
    float4 npos[DSR_NOALLOC_MAX_SLOTS];
    float4 nvel[DSR_NOALLOC_MAX_SLOTS];
    int32_t id[DSR_NOALLOC_MAX_SLOTS];
    int32_t partner[DSR_NOALLOC_MAX_SLOTS];
    dsr_u64 step;
};

__global__ void k_set_u64(dsr_u64* p, dsr_u64 v) { *p = v; }

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
NoallocScratch* g_noalloc_addr[kMaxDevices] = {};
}  // namespace

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// Device address of the scratch array on the current device. Host code may
// not use g_noalloc_scratch itself (its host-side name is a stand-in, not a
// device address); the address is looked up once per device, with that
// device current, and cached.
static int noalloc_scratch(int device, NoallocScratch** out) {
    if (device < 0 || device >= kMaxDevices) return DSR_E_INVALID;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            dsr__set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
            return DSR_E_CUDA;
        }
        g_noalloc_addr[device] = static_cast<NoallocScratch*>(p);
    }
    *out = g_noalloc_addr[device];
    return DSR_OK;
}

extern "C" int dsr_nbody_step_noalloc(dsr_heap* heap, const dsr_nbody_params* p, int n_steps, uint64_t step0,
                                      void* log_dev, uint64_t log_cap, void* log_count_dev, void* stream) {
    if (!heap || !p || n_steps < 0 || !log_count_dev || (log_cap && !log_dev) || !heap_matches(heap))
        return DSR_E_INVALID;
    const uint64_t S = heap->layout.n_blocks * 64;
    if (S > DSR_NOALLOC_MAX_SLOTS) return DSR_E_TOO_LARGE;
    int device = -1;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) {
        dsr__set_cuda_error(e, "dsr_nbody_step_noalloc");
        return DSR_E_CUDA;
    }
    if (device != heap->device) return DSR_E_INVALID;
    NoallocScratch* sc = nullptr;
    int rc = noalloc_scratch(device, &sc);
    if (rc) return rc;
    NbArgs a;
    a.p = *p;
    a.ws.pos = sc->pos;
    a.ws.npos = sc->npos;
    a.ws.nvel = sc->nvel;
    a.ws.id = sc->id;
    a.ws.partner = sc->partner;
    a.ws.step = &sc->step;
    a.ws.part = nullptr;  // the unsplit kernels below need no slice buffers
    a.ws.pbest = nullptr;
    a.ws.log = static_cast<int32_t*>(log_dev);
    a.ws.log_n = static_cast<dsr_u64*>(log_count_dev);
    a.ws.log_cap = log_cap;
    cudaStream_t s = dsr__stream(stream);
    // The array keeps the previous call's contents; the step counter is the
    // only value a step reads before writing it.
    k_set_u64<<<1, 1, 0, s>>>(&sc->step, step0);
    dsr_heap* h = heap;
    const unsigned dense_ctas = (unsigned)((S + TILE - 1) / TILE);
    const unsigned stream_ctas = (unsigned)(h->sm_count * 4);
    for (int i = 0; i < n_steps; ++i) {
        dsr__launch_scan(h, BODY, s);
        k_gather<<<stream_ctas, 256, 0, s>>>(h->dev, a.ws);
        k_force<<<dense_ctas, TILE, 0, s>>>(h->dev, a);
        k_partner<<<dense_ctas, TILE, 0, s>>>(h->dev, a);
        k_merge<<<stream_ctas, 256, 0, s>>>(h->dev, a);
    }
    return dsr__check_launch("dsr_nbody_step_noalloc");
}
