// N-body with merging collisions as an SMMO program (Fig. 6b "collisions"
// and 6d "nbody"; Fig. 1 names an Euler time step).
//
// One step is a do-all over Body whose block list R is built once and shared
// by the step's kernels (no body is created or deleted until the last one):
//   gather   each listed slot writes its body's state to dense arrays indexed
//            by g = R index * 64 + slot (empty slots: mass 0);
//   force    a_i = G sum_j m_j d_ij / (|d_ij|^2 + eps^2)^(3/2) over all dense
//            entries, tiled through shared memory;
//   update   v += a dt, x += v dt (semi-implicit Euler), written to the
//            object and to the dense arrays of the updated state;
//   partner  on the updated positions, the partner of i is the body with the
//            lowest id j != i within r_merge;
//   merge    mutual partners merge: the lower id takes the summed mass and
//            the mass-weighted position and velocity, the higher id deletes
//            itself.
// The last kernel's last CTA resets R.
//
// Precision. The state is stored as FP32 pairs: each of x, y, z, vx, vy, vz
// and m is a high word (its FP32 value) and a low word (the FP32 rounding of
// what the high word misses), about 48 significant bits together. The O(N)
// update, the merge-partner distance test and the merges run in FP64. The
// all-pairs interaction, the O(N^2) work, runs in one of two modes:
//   FP32 pairs  the sum runs in FP32 on the high words, except for pairs
//               closer than r_near (an FP32 test on the high words decides),
//               which are left out of it and added in FP64 from the full
//               state, in the order of the partners' ids;
//   FP64 pairs  every pair in FP64 from the full state.
// Close encounters amplify whatever error a step makes: rounding the stored
// positions to FP32 alone gives two bodies 2e-3 apart a separation error of
// about 3e-5 relative each step, which the next encounter multiplies; FP32
// far-field rounding, about 1e-9 of a close pair's relative acceleration,
// grows the same way over tens of steps.
#include <cfloat>
#include "dsr_apps.h"
#include "dsr_internal.cuh"

#include <mutex>

namespace {
enum { BODY = 0 };
enum { ID = 0, PX = 1, PY = 2, PZ = 3, VX = 4, VY = 5, VZ = 6, MASS = 7 };
constexpr int LO = 7;  // field f's low word is field f + LO (f = PX .. MASS)
constexpr int N_FIELDS = 15;
constexpr int TILE = 256;

// Four doubles in one 32-byte aligned record (x, y, z, m or vx, vy, vz, 0).
struct __align__(32) D4 {
    double x, y, z, w;
};
__device__ __forceinline__ D4 d4(double x, double y, double z, double w) { return D4{x, y, z, w}; }

struct NbWs {
    float4* pos;       // [S] high words x, y, z, m before the update (m = 0: empty slot)
    D4* pd;            // [S] full x, y, z, m before the update
    float4* npos;      // [S] high words x, y, z, m after the update
    D4* npd;           // [S] full x, y, z, m after the update
    D4* nvd;           // [S] full vx, vy, vz after the update
    int32_t* id;       // [S] body id, INT_MAX for an empty slot
    int32_t* partner;  // [S] dense index of the partner, -1 if none
    float4* part;      // [ns][stride] FP32 far-field sums per slice of j tiles
    D4* part64;        // [ns][stride] FP64 sums per slice (FP64 pairs; the same bytes as part)
    int2* pbest;       // [ns][stride] lowest partner id and its index per slice (split kernels)
    uint32_t* ncnt;    // [S] near pairs of body g
    uint32_t* noff;    // [S + 1] exclusive prefix sum of ncnt
    uint32_t* ncur;    // [S] fill cursors
    int2* pairs;       // [pair_cap] near pairs (i, j), in the order they were found
    int32_t* csr;      // [pair_cap] j of the near pairs, grouped by i
    uint32_t* npairs;  // near pairs found this step
    int32_t* log;      // [log_cap][3] merges: step, survivor id, absorbed id
    dsr_u64* log_n;    // merges logged so far
    dsr_u64* step;     // device step counter
    dsr_u64 log_cap;
    uint32_t pair_cap;
};

struct NbArgs {
    NbWs ws;
    dsr_nbody_params p;
};

__device__ __forceinline__ float* fld(const dsr_dev_heap& H, dsr_ref r, int f) { return dsr_field<float>(H, BODY, r, f); }

// Full value of a stored FP32 pair (high word f, low word f + LO).
__device__ __forceinline__ double get2(const dsr_dev_heap& H, dsr_ref r, int f) {
    return (double)*fld(H, r, f) + (double)*fld(H, r, f + LO);
}
// Store v as an FP32 pair: the high word is v rounded to FP32, the low word
// the FP32 rounding of the remainder (computed exactly in FP64).
__device__ __forceinline__ void put2(const dsr_dev_heap& H, dsr_ref r, int f, double v) {
    const float hi = __double2float_rn(v);
    *fld(H, r, f) = hi;
    *fld(H, r, f + LO) = __double2float_rn(v - (double)hi);
}

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

__device__ __forceinline__ bool slot_live(const dsr_dev_heap& H, uint32_t g) {
    return (H.R_mask[g >> 6] >> (g & 63)) & 1ull;
}
__device__ __forceinline__ dsr_ref slot_ref(const dsr_dev_heap& H, uint32_t g) {
    return ((dsr_u64)H.R_bid[g >> 6] << 6) | (g & 63);
}

__global__ void k_gather(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbWs ws) {
    const uint32_t n = n_dense(H);
    if (blockIdx.x == 0 && threadIdx.x == 0) *ws.npairs = 0;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        ws.ncnt[g] = 0;
        if (slot_live(H, g)) {
            const dsr_ref r = slot_ref(H, g);
            ws.pos[g] = make_float4(*fld(H, r, PX), *fld(H, r, PY), *fld(H, r, PZ), *fld(H, r, MASS));
            ws.pd[g] = d4(get2(H, r, PX), get2(H, r, PY), get2(H, r, PZ), get2(H, r, MASS));
            ws.id[g] = *dsr_field<int32_t>(H, BODY, r, ID);
        } else {
            ws.pos[g] = make_float4(0.f, 0.f, 0.f, 0.f);
            ws.pd[g] = d4(0.0, 0.0, 0.0, 0.0);
            ws.id[g] = 0x7FFFFFFF;
        }
    }
}

// 1/sqrt(x) by the PTX approximate reciprocal square root with subnormal
// inputs flushed to zero; used only where x >= eps^2 >= FLT_MIN (or +inf, for
// an excluded pair), so the flush never applies.
__device__ __forceinline__ float rsqrt_normal(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// A near pair (i, j), found by the thread of body i: recorded for the FP64
// near field. Returns false when the pair list is full (the pair then stays
// in the FP32 sum, and the heap's DSR_ERR_CAPACITY bit reports it).
__device__ __forceinline__ bool near_record(const dsr_dev_heap& H, const NbWs& ws, uint32_t gi, uint32_t gj) {
    const uint32_t k = atomicAdd(ws.npairs, 1u);
    if (k >= ws.pair_cap) {
        atomicOr(H.err, DSR_ERR_CAPACITY);
        return false;
    }
    ws.pairs[k] = make_int2((int)gi, (int)gj);
    atomicAdd(ws.ncnt + gi, 1u);
    return true;
}

// The rare branch of the force kernels: body gi lies within r_near of body
// gj. The pair is recorded for the FP64 near field and must then be left out
// of the FP32 sum (true); so must the body itself, whose term is 0 either
// way. False: the pair stays in the FP32 sum (an empty slot, or a full list).
__device__ __forceinline__ bool near_pair(const dsr_dev_heap& H, const NbWs& ws, uint32_t gi, uint32_t gj, float mj,
                                          uint32_t n) {
    if (gi == gj) return true;
    if (gi >= n || mj <= 0.f || ws.pos[gi].w <= 0.f) return false;
    return near_record(H, ws, gi, gj);
}

__device__ __forceinline__ float f_inf() { return __int_as_float(0x7F800000); }

// Split all-pairs kernels, the ones dsr_nbody_step runs.
//
// Work items. A row item is TILE * RB bodies (RB per thread), the j tiles are
// cut into `ns` slices, and a work item is one (row item, slice) pair; `ns`
// follows from the dense count on the device (n_slices), so the items fill
// about `grid` CTAs whatever the live count. Each item writes its partial
// result to part[slice][g] (pbest for the partner search); the update and the
// partner combine read the slices back in slice order, so the result does not
// depend on which CTA ran which item.
//
// Register blocking. Every lane of a warp reads the same j body from shared
// memory (a broadcast), and at one body per thread the shared-memory return
// path, not the FP32 pipe, sets the pace. With RB bodies per thread each
// load feeds RB pairs.
constexpr int RB = 4;  // bodies per thread in the split kernels

__device__ __forceinline__ uint32_t n_slices(uint32_t nr, uint32_t nj, uint32_t grid) {
    if (!nr) return 0;
    const uint32_t k = grid / nr;
    return k < 1 ? 1 : (k > nj ? nj : k);
}

constexpr int RB64 = 2;  // bodies per thread in the FP64 kernel

struct SplitShape {
    uint32_t n, nj, nr, ns;  // dense count, j tiles, row items, slices
};

// Work items of a split kernel with rb bodies per thread.
__device__ __forceinline__ SplitShape split_shape(const dsr_dev_heap& H, uint32_t grid, int rb = RB) {
    SplitShape q;
    q.n = n_dense(H);
    q.nj = (q.n + TILE - 1) / TILE;
    q.nr = (q.n + TILE * rb - 1) / (TILE * rb);
    q.ns = n_slices(q.nr, q.nj, grid);
    return q;
}

// FP32 far-field sums of one slice of j tiles for RB bodies per thread (body
// k of a thread: row * TILE * RB + k * TILE + threadIdx.x), Kahan-compensated
// across tiles. A pair within r_near goes to the near field (near_pair, a
// branch that almost never runs: one compare per pair on the common path).
// SOFT: eps^2 >= FLT_MIN, so r^2 >= eps^2 is a normal number for every pair,
// the body itself included, and no zero-distance guard is needed.
template <bool SOFT>
__global__ void __launch_bounds__(TILE) k_force_part(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbArgs a) {
    __shared__ float4 sp[TILE];
    const SplitShape q = split_shape(H, gridDim.x);
    const float eps2 = (float)(a.p.eps * a.p.eps);
    const float rn2 = (float)(a.p.r_near * a.p.r_near);
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
                    float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                    if (r2 < rn2 && near_pair(H, a.ws, g0 + k * TILE, t * TILE + j, pj.w, q.n)) r2 = f_inf();
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

// Unsplit force kernel (the allocation-free step): one thread per dense slot,
// one CTA per TILE slots, the same pair arithmetic and near-field rule as
// k_force_part. The sums go to part[g] (a single slice).
__global__ void __launch_bounds__(TILE) k_force(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbArgs a) {
    __shared__ float4 sp[TILE];
    const uint32_t n = n_dense(H);
    const uint32_t base = blockIdx.x * TILE;
    if (base >= n) return;
    const uint32_t g = base + threadIdx.x;
    const float4 pi = ws_load(a.ws.pos, g, n);
    const float eps2 = (float)(a.p.eps * a.p.eps);
    const float rn2 = (float)(a.p.r_near * a.p.r_near);
    float ax = 0.f, ay = 0.f, az = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    for (uint32_t t0 = 0; t0 < n; t0 += TILE) {
        __syncthreads();
        sp[threadIdx.x] = ws_load(a.ws.pos, t0 + threadIdx.x, n);
        __syncthreads();
        float tx = 0.f, ty = 0.f, tz = 0.f;
        for (int j = 0; j < TILE; ++j) {
            const float4 pj = sp[j];
            const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
            if (r2 < rn2 && near_pair(H, a.ws, g, t0 + j, pj.w, n)) r2 = f_inf();
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
    if (g < n) a.ws.part[g] = make_float4(ax, ay, az, 0.f);
}

__device__ __forceinline__ D4 ws_load64(const D4* p, uint32_t g, uint32_t n) {
    return g < n ? p[g] : d4(0.0, 0.0, 0.0, 0.0);
}

// One FP64 pair term added to (ax, ay, az): body j at pj acting on a body at
// (px, py, pz). A zero r^2 (a body on itself with eps = 0) adds nothing.
__device__ __forceinline__ void pair64(const D4& pj, double px, double py, double pz, double eps2, double& ax,
                                       double& ay, double& az) {
    const double dx = pj.x - px, dy = pj.y - py, dz = pj.z - pz;
    const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    const double inv = r2 > 0.0 ? rsqrt(r2) : 0.0;
    const double w = pj.w * inv * inv * inv;
    ax = fma(w, dx, ax);
    ay = fma(w, dy, ay);
    az = fma(w, dz, az);
}

// FP64 pairs, split form: as k_force_part with RB64 bodies per thread, every
// pair in FP64 from the full state; sums per slice in part64.
__global__ void __launch_bounds__(TILE) k_force_part64(const __grid_constant__ dsr_dev_heap H,
                                                       const __grid_constant__ NbArgs a) {
    __shared__ D4 sp[TILE];
    const SplitShape q = split_shape(H, gridDim.x, RB64);
    const double eps2 = a.p.eps * a.p.eps;
    for (uint32_t item = blockIdx.x; item < q.nr * q.ns; item += gridDim.x) {
        const uint32_t row = item % q.nr, sl = item / q.nr;
        const uint32_t g0 = row * TILE * RB64 + threadIdx.x;
        double px[RB64], py[RB64], pz[RB64], ax[RB64], ay[RB64], az[RB64];
#pragma unroll
        for (int k = 0; k < RB64; ++k) {
            const D4 u = ws_load64(a.ws.pd, g0 + k * TILE, q.n);
            px[k] = u.x, py[k] = u.y, pz[k] = u.z;
            ax[k] = ay[k] = az[k] = 0.0;
        }
        for (uint32_t t = q.nj * sl / q.ns; t < q.nj * (sl + 1) / q.ns; ++t) {
            __syncthreads();
            sp[threadIdx.x] = ws_load64(a.ws.pd, t * TILE + threadIdx.x, q.n);
            __syncthreads();
#pragma unroll 2
            for (int j = 0; j < TILE; ++j) {
                const D4 pj = sp[j];
#pragma unroll
                for (int k = 0; k < RB64; ++k) pair64(pj, px[k], py[k], pz[k], eps2, ax[k], ay[k], az[k]);
            }
        }
        D4* out = a.ws.part64 + (size_t)sl * q.nr * TILE * RB64;
#pragma unroll
        for (int k = 0; k < RB64; ++k)
            if (g0 + k * TILE < q.n) out[g0 + k * TILE] = d4(ax[k], ay[k], az[k], 0.0);
    }
}

// FP64 pairs, unsplit (the allocation-free step): one thread per dense slot.
__global__ void __launch_bounds__(TILE) k_force64(const __grid_constant__ dsr_dev_heap H,
                                                  const __grid_constant__ NbArgs a) {
    __shared__ D4 sp[TILE];
    const uint32_t n = n_dense(H);
    const uint32_t base = blockIdx.x * TILE;
    if (base >= n) return;
    const uint32_t g = base + threadIdx.x;
    const D4 pi = ws_load64(a.ws.pd, g, n);
    const double eps2 = a.p.eps * a.p.eps;
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (uint32_t t0 = 0; t0 < n; t0 += TILE) {
        __syncthreads();
        sp[threadIdx.x] = ws_load64(a.ws.pd, t0 + threadIdx.x, n);
        __syncthreads();
        for (int j = 0; j < TILE; ++j) pair64(sp[j], pi.x, pi.y, pi.z, eps2, ax, ay, az);
    }
    if (g < n) a.ws.part64[g] = d4(ax, ay, az, 0.0);
}

// Exclusive prefix sum of the near-pair counts (one CTA of 1024 threads, each
// summing a contiguous run of bodies), and the fill cursors cleared.
__global__ void __launch_bounds__(1024) k_near_scan(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbWs ws) {
    __shared__ uint32_t part[1024];
    const uint32_t n = n_dense(H);
    const uint32_t per = (n + 1023) / 1024;
    const uint32_t lo = threadIdx.x * per, hi = lo + per < n ? lo + per : n;
    uint32_t s = 0;
    for (uint32_t g = lo; g < hi; ++g) s += ws.ncnt[g];
    part[threadIdx.x] = s;
    __syncthreads();
    for (uint32_t d = 1; d < 1024; d <<= 1) {  // inclusive scan of the run sums
        const uint32_t v = threadIdx.x >= d ? part[threadIdx.x - d] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - s;
    for (uint32_t g = lo; g < hi; ++g) {
        ws.noff[g] = run;
        ws.ncur[g] = 0;
        run += ws.ncnt[g];
    }
    if (threadIdx.x == 1023) ws.noff[n] = part[1023];
}

// Near pairs grouped by their body i (in arbitrary order within a group; the
// update sorts each group by the partners' ids).
__global__ void k_near_fill(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbWs ws) {
    (void)H;
    uint32_t m = *ws.npairs;
    if (m > ws.pair_cap) m = ws.pair_cap;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        const int2 p = ws.pairs[k];
        ws.csr[ws.noff[p.x] + atomicAdd(ws.ncur + p.x, 1u)] = p.y;
    }
}

// The update of body g: the FP32 far-field slices summed in slice order (in
// FP64), the near field in FP64 over the partners sorted by id, then
// v += a dt and x += v dt on the full state, stored back as FP32 pairs.
__device__ void update_body(const dsr_dev_heap& H, const NbArgs& a, uint32_t g, uint32_t ns, size_t stride,
                            bool f64) {
    const dsr_ref r = slot_ref(H, g);
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (uint32_t k = 0; k < ns; ++k) {
        if (f64) {
            const D4 v = a.ws.part64[k * stride + g];
            ax += v.x;
            ay += v.y;
            az += v.z;
        } else {
            const float4 v = a.ws.part[k * stride + g];
            ax += (double)v.x;
            ay += (double)v.y;
            az += (double)v.z;
        }
    }
    const D4 pi = a.ws.pd[g];
    const double eps2 = a.p.eps * a.p.eps;
    int32_t* seg = a.ws.csr + a.ws.noff[g];
    const uint32_t cnt = a.ws.noff[g + 1] - a.ws.noff[g];
    for (uint32_t u = 1; u < cnt; ++u) {  // insertion sort by id (ids are unique)
        const int32_t x = seg[u];
        const int32_t key = a.ws.id[x];
        uint32_t v = u;
        while (v > 0 && a.ws.id[seg[v - 1]] > key) {
            seg[v] = seg[v - 1];
            --v;
        }
        seg[v] = x;
    }
    for (uint32_t u = 0; u < cnt; ++u) {
        const D4 pj = a.ws.pd[seg[u]];
        const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        const double r2 = dx * dx + dy * dy + dz * dz + eps2;
        const double w = pj.w / (r2 * sqrt(r2));
        ax += w * dx;
        ay += w * dy;
        az += w * dz;
    }
    const double G = a.p.G, dt = a.p.dt;
    const double vx = get2(H, r, VX) + G * ax * dt;
    const double vy = get2(H, r, VY) + G * ay * dt;
    const double vz = get2(H, r, VZ) + G * az * dt;
    const double x = pi.x + vx * dt, y = pi.y + vy * dt, z = pi.z + vz * dt;
    put2(H, r, VX, vx);
    put2(H, r, VY, vy);
    put2(H, r, VZ, vz);
    put2(H, r, PX, x);
    put2(H, r, PY, y);
    put2(H, r, PZ, z);
    a.ws.npos[g] = make_float4(*fld(H, r, PX), *fld(H, r, PY), *fld(H, r, PZ), *fld(H, r, MASS));
    a.ws.npd[g] = d4(x, y, z, pi.w);
    a.ws.nvd[g] = d4(vx, vy, vz, 0.0);
}

// Update of every live body; `grid` is the split force kernel's grid (0: the
// unsplit kernel's single slice).
__global__ void k_update(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbArgs a, uint32_t grid) {
    const bool f64 = a.p.pair_precision == DSR_NBODY_PAIRS_FP64;
    const int rb = f64 ? RB64 : RB;
    uint32_t ns = 1;
    size_t stride = 0;
    if (grid) {
        const SplitShape q = split_shape(H, grid, rb);
        ns = q.ns;
        stride = (size_t)q.nr * TILE * rb;
    }
    const uint32_t n = n_dense(H);
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        if (slot_live(H, g))
            update_body(H, a, g, ns, stride, f64);
        else
            a.ws.npos[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Merge-partner test of body gi against gj, both with updated positions:
// the FP32 test on the high words, widened by `rw2`, selects candidates; the
// decision is the FP64 distance on the full positions against r_merge.
__device__ __forceinline__ bool within_merge(const NbArgs& a, uint32_t gi, uint32_t gj) {
    const D4 u = a.ws.npd[gi], v = a.ws.npd[gj];
    const double dx = v.x - u.x, dy = v.y - u.y, dz = v.z - u.z;
    return dx * dx + dy * dy + dz * dz < a.p.r_merge * a.p.r_merge;
}

// FP32 radius that selects merge candidates: r_merge plus a margin above the
// rounding of the high words (positions of magnitude below 64).
__device__ __forceinline__ float wide_merge2(const NbArgs& a) {
    const float rw = (float)(a.p.r_merge * (1.0 + 1e-3) + 1e-5);
    return rw * rw;
}

// Partner search over one slice of j tiles for RB bodies per thread: per
// body the lowest partner id in the slice and that partner's dense index.
// The candidate test fails for almost every pair, so the common path is the
// squared distances and one test of their minimum; the per-body tests, the
// FP64 decision and the id sit behind it.
__global__ void __launch_bounds__(TILE, 5) k_partner_part(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbArgs a) {
    __shared__ float4 sp[TILE];
    const SplitShape q = split_shape(H, gridDim.x);
    const float rw2 = wide_merge2(a);
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
                if (dmin < rw2 && pj.w > 0.f) {
                    const uint32_t jg = t0 + j;
#pragma unroll
                    for (int k = 0; k < RB; ++k) {
                        const uint32_t gk = g0 + k * TILE;
                        if (d2[k] < rw2 && jg != gk && gk < q.n) {
                            const int32_t jid = a.ws.id[jg];
                            if (jid < best_id[k] && within_merge(a, gk, jg)) {
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
__global__ void k_partner_combine(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbArgs a, uint32_t grid) {
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

// Unsplit partner search (the allocation-free step): lowest id within
// r_merge, with the candidate test and FP64 decision of k_partner_part.
__global__ void __launch_bounds__(TILE) k_partner(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbArgs a) {
    __shared__ float4 sp[TILE];
    __shared__ int32_t sid[TILE];
    const uint32_t n = n_dense(H);
    const uint32_t base = blockIdx.x * TILE;
    if (base >= n) return;
    const uint32_t g = base + threadIdx.x;
    const float4 pi = g < n ? a.ws.npos[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float rw2 = wide_merge2(a);
    int32_t best_id = 0x7FFFFFFF, best = -1;
    for (uint32_t t0 = 0; t0 < n; t0 += TILE) {
        __syncthreads();
        const uint32_t j = t0 + threadIdx.x;
        sp[threadIdx.x] = j < n ? a.ws.npos[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        sid[threadIdx.x] = j < n ? a.ws.id[j] : 0x7FFFFFFF;
        __syncthreads();
        for (int k = 0; k < TILE; ++k) {
            const float4 pj = sp[k];
            const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const int32_t jid = sid[k];
            if (d2 < rw2 && jid < best_id && t0 + k != g && pj.w > 0.f && g < n && within_merge(a, g, t0 + k)) {
                best_id = jid;
                best = (int32_t)(t0 + k);
            }
        }
    }
    if (g < n) a.ws.partner[g] = (pi.w > 0.f) ? best : -1;
}

// Merge mutual partners in FP64; the higher id deletes itself. Last kernel
// of the step: its last CTA resets R and advances the step counter.
__global__ void k_merge(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbArgs a) {
    const uint32_t n = n_dense(H);
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t g = base + threadIdx.x;
        if (g >= n) continue;
        const int32_t j = a.ws.partner[g];
        if (j < 0 || a.ws.partner[j] != (int32_t)g) continue;
        const dsr_ref r = slot_ref(H, g);
        if (a.ws.id[g] > a.ws.id[j]) {
            dsr_delete(H, r);
            continue;
        }
        const D4 pg = a.ws.npd[g], pj = a.ws.npd[j];
        const D4 vg = a.ws.nvd[g], vj = a.ws.nvd[j];
        const double M = pg.w + pj.w;
        put2(H, r, VX, (pg.w * vg.x + pj.w * vj.x) / M);
        put2(H, r, VY, (pg.w * vg.y + pj.w * vj.y) / M);
        put2(H, r, VZ, (pg.w * vg.z + pj.w * vj.z) / M);
        put2(H, r, PX, (pg.w * pg.x + pj.w * pj.x) / M);
        put2(H, r, PY, (pg.w * pg.y + pj.w * pj.y) / M);
        put2(H, r, PZ, (pg.w * pg.z + pj.w * pj.z) / M);
        put2(H, r, MASS, M);
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
        for (int f = 0; f < 7; ++f) {
            *fld(H, r, PX + f) = rows[7 * i + f];
            *fld(H, r, PX + f + LO) = 0.f;
        }
    }
}

const int kBodyFields[N_FIELDS] = {4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4};

bool heap_matches(const dsr_heap* h) {
    const dsr_layout& L = h->layout;
    if (L.n_types < 1 || L.n_fields[BODY] != N_FIELDS) return false;
    for (int f = 0; f < N_FIELDS; ++f)
        if (L.field_bytes[BODY][f] != 4) return false;
    return true;
}

bool params_ok(const dsr_nbody_params* p) {
    return p && p->dt > 0.0 && p->eps >= 0.0 && p->r_merge >= 0.0 && p->r_near >= 0.0 &&
           p->r_near * p->r_near < (double)FLT_MAX && p->r_merge * p->r_merge < (double)FLT_MAX &&
           (p->pair_precision == DSR_NBODY_PAIRS_FP32 || p->pair_precision == DSR_NBODY_PAIRS_FP64);
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Grid of a split all-pairs kernel: four waves of its resident CTAs.
uint32_t split_grid(const dsr_heap* h, const void* kernel) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, TILE, 0) != cudaSuccess || occ < 1) occ = 1;
    return (uint32_t)(4 * occ * h->sm_count);
}

struct SplitGrids {
    uint32_t force, force64, partner;
};

SplitGrids split_grids(const dsr_heap* h) {
    return {split_grid(h, (const void*)k_force_part<true>), split_grid(h, (const void*)k_force_part64),
            split_grid(h, (const void*)k_partner_part)};
}

// Slice entries of a split kernel: ns * nr <= max(grid, nr) items of TILE * rb bodies.
size_t slots_for(uint64_t S, uint32_t grid, int rb) {
    const uint64_t nr = (S + TILE * rb - 1) / (TILE * rb);
    return (size_t)(grid > nr ? grid : nr) * TILE * rb;
}
size_t split_slots(uint64_t S, SplitGrids g) {
    const size_t a = slots_for(S, g.force, RB), b = slots_for(S, g.partner, RB);
    return a > b ? a : b;
}
// Bytes of the force slice buffer: FP32 sums (16 bytes a slot) or FP64 sums
// (32 bytes a slot, RB64 bodies a thread), whichever needs more.
size_t part_bytes(uint64_t S, SplitGrids g) {
    const size_t a = slots_for(S, g.force, RB) * 16, b = slots_for(S, g.force64, RB64) * 32;
    return a > b ? a : b;
}

// Near pairs a workspace holds: 32 per slot, at least 2^20.
uint64_t pair_cap_for(uint64_t S) { return S * 32 > (1u << 20) ? S * 32 : (1u << 20); }

// Dense per-slot arrays of a step for S slots, carved from p (advanced).
void carve_dense(uint8_t*& p, uint64_t S, NbWs& w) {
    w.pos = reinterpret_cast<float4*>(p);
    p += round256(S * 16);
    w.pd = reinterpret_cast<D4*>(p);
    p += round256(S * 32);
    w.npos = reinterpret_cast<float4*>(p);
    p += round256(S * 16);
    w.npd = reinterpret_cast<D4*>(p);
    p += round256(S * 32);
    w.nvd = reinterpret_cast<D4*>(p);
    p += round256(S * 32);
    w.id = reinterpret_cast<int32_t*>(p);
    p += round256(S * 4);
    w.partner = reinterpret_cast<int32_t*>(p);
    p += round256(S * 4);
    w.ncnt = reinterpret_cast<uint32_t*>(p);
    p += round256(S * 4);
    w.noff = reinterpret_cast<uint32_t*>(p);
    p += round256((S + 1) * 4);
    w.ncur = reinterpret_cast<uint32_t*>(p);
    p += round256(S * 4);
}
size_t dense_bytes(uint64_t S) {
    return 2 * round256(S * 16) + 3 * round256(S * 32) + 4 * round256(S * 4) + round256((S + 1) * 4);
}

size_t ws_bytes(uint64_t S, uint64_t log_cap, SplitGrids grid) {
    const uint64_t pc = pair_cap_for(S);
    return dense_bytes(S) + round256(pc * 8) + round256(pc * 4) + round256(log_cap * 12) + 256 +
           round256(part_bytes(S, grid)) + round256(split_slots(S, grid) * 8);
}

NbWs carve(void* base, uint64_t S, uint64_t log_cap, SplitGrids grid) {
    uint8_t* p = static_cast<uint8_t*>(base);
    NbWs w;
    carve_dense(p, S, w);
    const uint64_t pc = pair_cap_for(S);
    w.pairs = reinterpret_cast<int2*>(p);
    p += round256(pc * 8);
    w.csr = reinterpret_cast<int32_t*>(p);
    p += round256(pc * 4);
    w.pair_cap = (uint32_t)pc;
    w.log = reinterpret_cast<int32_t*>(p);
    p += round256(log_cap * 12);
    w.log_n = reinterpret_cast<dsr_u64*>(p);
    w.step = reinterpret_cast<dsr_u64*>(p + 8);
    w.npairs = reinterpret_cast<uint32_t*>(p + 16);
    p += 256;
    w.part = reinterpret_cast<float4*>(p);
    w.part64 = reinterpret_cast<D4*>(p);
    p += round256(part_bytes(S, grid));
    w.pbest = reinterpret_cast<int2*>(p);
    w.log_cap = log_cap;
    return w;
}

// The kernels between the force sums and the merge that both forms share:
// the near-pair grouping, the update (grid: the split force grid, or 0 for a
// single slice), then the partner search and the merge.
void launch_near_update(dsr_heap* h, const NbArgs& a, uint32_t grid, cudaStream_t s) {
    const unsigned stream_ctas = (unsigned)(h->sm_count * 4);
    k_near_scan<<<1, 1024, 0, s>>>(h->dev, a.ws);
    k_near_fill<<<stream_ctas, 256, 0, s>>>(h->dev, a.ws);
    k_update<<<stream_ctas, 256, 0, s>>>(h->dev, a, grid);
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
    out[0] = dsr_type_desc{"Body", N_FIELDS, kBodyFields};
    return DSR_OK;
}

extern "C" int dsr_nbody_workspace_bytes(const dsr_heap* heap, uint64_t log_cap, size_t* out) {
    if (!heap || !out) return DSR_E_INVALID;
    *out = ws_bytes(heap->layout.n_blocks * 64, log_cap, split_grids(heap));
    return DSR_OK;
}

extern "C" int dsr_nbody_create(dsr_heap* heap, const dsr_nbody_params* p, const void* rows_dev, int n_bodies,
                                void* workspace_dev, uint64_t log_cap, void* stream, dsr_nbody** out) {
    if (!heap || !params_ok(p) || !rows_dev || !workspace_dev || !out || n_bodies < 1) return DSR_E_INVALID;
    if ((reinterpret_cast<uintptr_t>(workspace_dev) & 255) || !heap_matches(heap)) return DSR_E_INVALID;
    if ((uint64_t)n_bodies > heap->layout.n_blocks * heap->layout.capacity[BODY]) return DSR_E_INVALID;
    const uint64_t S = heap->layout.n_blocks * 64;
    if (pair_cap_for(S) > 0xFFFFFFFFull) return DSR_E_INVALID;
    dsr_nbody* nb = new dsr_nbody;
    nb->heap = heap;
    nb->S = S;
    nb->grid = split_grids(heap);
    nb->args.ws = carve(workspace_dev, nb->S, log_cap, nb->grid);
    nb->args.p = *p;
    cudaStream_t s = dsr__stream(stream);
    cudaError_t e = cudaMemsetAsync(nb->args.ws.log_n, 0, 24, s);
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
    const bool soft = nb->args.p.eps * nb->args.p.eps >= (double)FLT_MIN;
    const bool f64 = nb->args.p.pair_precision == DSR_NBODY_PAIRS_FP64;
    for (int i = 0; i < n_steps; ++i) {
        dsr__launch_scan(h, BODY, s);
        k_gather<<<stream_ctas, 256, 0, s>>>(h->dev, nb->args.ws);
        if (f64)
            k_force_part64<<<nb->grid.force64, TILE, 0, s>>>(h->dev, nb->args);
        else if (soft)
            k_force_part<true><<<nb->grid.force, TILE, 0, s>>>(h->dev, nb->args);
        else
            k_force_part<false><<<nb->grid.force, TILE, 0, s>>>(h->dev, nb->args);
        launch_near_update(h, nb->args, f64 ? nb->grid.force64 : nb->grid.force, s);
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

extern "C" int dsr_nbody_near_pairs(dsr_nbody* nb, void** count_dev) {
    if (!nb || !count_dev) return DSR_E_INVALID;
    *count_dev = nb->args.ws.npairs;
    return DSR_OK;
}

extern "C" int dsr_nbody_destroy(dsr_nbody* nb) {
    delete nb;
    return DSR_OK;
}

int dsr__nbody_method(dsr_heap*, int, int, const void*, size_t, cudaStream_t, bool) { return DSR_E_INVALID; }

// ---------------------------------------------------------------------------
// Allocation-free step. The per-slot scratch of a step (the dense state
// before and after the update, ids, partners, the far-field sums and the
// near-pair lists) lives in this file-scope device array instead of a
// caller-allocated workspace, for callers that cannot call cudaMalloc.
// Every GPU that loads the library holds the array until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr uint64_t kNoallocPairs = (uint64_t)DSR_NOALLOC_MAX_SLOTS * DSR_NOALLOC_PAIRS_PER_SLOT;

struct NoallocScratch {
    float4 pos[DSR_NOALLOC_MAX_SLOTS];
    D4 pd[DSR_NOALLOC_MAX_SLOTS];
    float4 npos[DSR_NOALLOC_MAX_SLOTS];
    D4 npd[DSR_NOALLOC_MAX_SLOTS];
    D4 nvd[DSR_NOALLOC_MAX_SLOTS];
    D4 part[DSR_NOALLOC_MAX_SLOTS];  // far-field sums: FP32 (as float4) or FP64
    int32_t id[DSR_NOALLOC_MAX_SLOTS];
    int32_t partner[DSR_NOALLOC_MAX_SLOTS];
    uint32_t ncnt[DSR_NOALLOC_MAX_SLOTS];
    uint32_t noff[DSR_NOALLOC_MAX_SLOTS + 1];
    uint32_t ncur[DSR_NOALLOC_MAX_SLOTS];
    int2 pairs[kNoallocPairs];
    int32_t csr[kNoallocPairs];
    uint32_t npairs;
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
    if (!heap || !params_ok(p) || n_steps < 0 || !log_count_dev || (log_cap && !log_dev) || !heap_matches(heap))
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
    a.ws.pd = sc->pd;
    a.ws.npos = sc->npos;
    a.ws.npd = sc->npd;
    a.ws.nvd = sc->nvd;
    a.ws.part = reinterpret_cast<float4*>(sc->part);  // one slice: the unsplit force kernels
    a.ws.part64 = sc->part;
    a.ws.pbest = nullptr;  // the unsplit partner kernel needs no slice buffer
    a.ws.id = sc->id;
    a.ws.partner = sc->partner;
    a.ws.ncnt = sc->ncnt;
    a.ws.noff = sc->noff;
    a.ws.ncur = sc->ncur;
    a.ws.pairs = sc->pairs;
    a.ws.csr = sc->csr;
    a.ws.pair_cap = (uint32_t)kNoallocPairs;
    a.ws.npairs = &sc->npairs;
    a.ws.step = &sc->step;
    a.ws.log = static_cast<int32_t*>(log_dev);
    a.ws.log_n = static_cast<dsr_u64*>(log_count_dev);
    a.ws.log_cap = log_cap;
    cudaStream_t s = dsr__stream(stream);
    // The array keeps the previous call's contents. The step counter is the
    // only value a step reads before this call writes it; the pair count and
    // the per-body counts are cleared by each step's gather.
    k_set_u64<<<1, 1, 0, s>>>(&sc->step, step0);
    dsr_heap* h = heap;
    const unsigned dense_ctas = (unsigned)((S + TILE - 1) / TILE);
    const unsigned stream_ctas = (unsigned)(h->sm_count * 4);
    for (int i = 0; i < n_steps; ++i) {
        dsr__launch_scan(h, BODY, s);
        k_gather<<<stream_ctas, 256, 0, s>>>(h->dev, a.ws);
        if (a.p.pair_precision == DSR_NBODY_PAIRS_FP64)
            k_force64<<<dense_ctas, TILE, 0, s>>>(h->dev, a);
        else
            k_force<<<dense_ctas, TILE, 0, s>>>(h->dev, a);
        launch_near_update(h, a, 0, s);
        k_partner<<<dense_ctas, TILE, 0, s>>>(h->dev, a);
        k_merge<<<stream_ctas, 256, 0, s>>>(h->dev, a);
    }
    return dsr__check_launch("dsr_nbody_step_noalloc");
}
