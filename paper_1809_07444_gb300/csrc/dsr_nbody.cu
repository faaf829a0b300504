// N-body with merging collisions as an SMMO program (Fig. 6b "collisions"
// and 6d "nbody"; Fig. 1 names an Euler time step).
//
// One step is a do-all over Body whose block list R is built once and shared
// by the step's kernels (no body is created or deleted until the last one).
// The live bodies are first put in spatial order: a counting sort by cell of
// a K^3 grid over the unit cube (positions outside it fall in the border
// cells), cells in Morton order, the bodies of a cell by id. On that order:
//   gather   sorted position p holds its body's state and handle; each tile
//            of 256 positions gets the bounding box of its bodies;
//   force    a_i = G sum_j m_j d_ij / (|d_ij|^2 + eps^2)^(3/2), all pairs,
//            tiled through shared memory (FP32 or FP64 pairs, below);
//   update   the far-field slices summed, the near field added (FP32 pairs:
//            pairs closer than r_near, found in the 27 cells around the
//            body's own, in FP64), then v += a dt, x += v dt (semi-implicit
//            Euler) in FP64, written to the object;
//   partner  the bodies are sorted again by the cells of their new
//            positions; the partner of i is the body with the lowest id
//            j != i within r_merge, found in the 27 cells around i's;
//   merge    mutual partners merge: the lower id takes the summed mass and
//            the mass-weighted position and velocity, the higher id deletes
//            itself.
// The last kernel's last CTA resets R. Every sum is taken in a fixed order
// (positions, tiles, slices, cells and ids), so a step is deterministic.
//
// Precision. The state is stored as FP32 pairs: each of x, y, z, vx, vy, vz
// and m is a high word (its FP32 value) and a low word (the FP32 rounding of
// what the high word misses), about 48 significant bits together. The O(N)
// update, the merge-partner distance test and the merges run in FP64. The
// all-pairs interaction, the O(N^2) work, runs in one of two modes:
//   FP32 pairs  the sum runs in FP32 on the high words, except for pairs
//               closer than r_near (an FP32 test on the high words decides),
//               which are left out of it and added in FP64 from the full
//               state;
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
constexpr int RB = 4;      // bodies per thread in the FP32 force kernel
constexpr int RB64 = 2;    // bodies per thread in the FP64 force kernel
constexpr int ROW = 1024;  // sorted positions are padded to a multiple of this (TILE * RB)
constexpr int KMAX = 32;   // cells per axis at most
constexpr uint32_t NKEYS = KMAX * KMAX * KMAX;  // Morton keys of 5-bit cell coordinates

// Four doubles in one 32-byte aligned record (x, y, z, m or vx, vy, vz, 0).
struct __align__(32) D4 {
    double x, y, z, w;
};
__device__ __forceinline__ D4 d4(double x, double y, double z, double w) { return D4{x, y, z, w}; }

struct NbWs {
    // spatial order
    uint32_t* ccount;  // [NKEYS] bodies per cell (zero between sorts)
    uint32_t* coff;    // [NKEYS + 1] first sorted position of each cell (positions before the update)
    uint32_t* coff2;   // [NKEYS + 1] the same for the positions after the update
    uint32_t* ckey;    // [P] cell key of each element being sorted
    uint32_t* csum;    // [NKEYS / 1024] cells per CTA of the prefix sum
    uint32_t* perm;    // [P] dense slot of each sorted position
    uint32_t* perm2;   // [P] sorted position of each entry of the second order
    uint32_t* n_live;  // bodies in this step
    uint32_t* npairs;  // near-field pairs of this step (each counted from both bodies)
    // per sorted position p (padded to a multiple of ROW with empty entries)
    float4* pos;       // high words x, y, z, m before the update (m = 0: empty)
    D4* pd;            // full x, y, z, m before the update
    int32_t* id;       // body id, INT_MAX for an empty entry
    dsr_u64* sref;     // the body's handle
    float4* tbox;      // [2 per tile] bounding box (low corner, high corner) of a tile's bodies
    float4* npos;      // high words x, y, z, m after the update
    D4* npd;           // full x, y, z, m after the update
    D4* nvd;           // full vx, vy, vz after the update
    int32_t* partner;  // sorted position of the partner, -1 if none
    float4* part;      // [ns][P] FP32 far-field sums per slice of j tiles
    D4* part64;        // [ns][P] FP64 sums per slice (FP64 pairs; the same bytes as part)
    int32_t* log;      // [log_cap][3] merges: step, survivor id, absorbed id
    dsr_u64* log_n;    // merges logged so far
    dsr_u64* step;     // device step counter
    dsr_u64 log_cap;
    int32_t K;         // cells per axis
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

// Compensated (Kahan) accumulation: s += x with the lost low part kept in c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Error-free sum (Knuth's TwoSum): s + x = t + err exactly, t = fl(s + x).
// Accumulating err in e keeps s + e within about 2^-43 relative of the exact
// sum of a few dozen FP32 terms, in FP32 arithmetic only.
__device__ __forceinline__ void two_sum_add(float& s, float& e, float x) {
    const float t = s + x;
    const float bp = t - s;
    e += (s - (t - bp)) + (x - bp);
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

__device__ __forceinline__ uint32_t n_bodies(const NbWs& ws) { return *(volatile uint32_t*)ws.n_live; }
// Sorted positions in use: the live bodies, padded to a whole row item.
__device__ __forceinline__ uint32_t n_padded(const NbWs& ws) { return (n_bodies(ws) + ROW - 1) / ROW * ROW; }

// ---------------------------------------------------------------------------
// spatial order
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_coord(float x, int K) {
    const float c = floorf(x * (float)K);  // monotone in x: bodies closer than a cell's width are in adjacent cells
    return c < 0.f ? 0 : (c >= (float)K ? K - 1 : (int)c);
}
__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // 5 bits to every third bit
    uint32_t r = 0;
#pragma unroll
    for (int b = 0; b < 5; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}
__device__ __forceinline__ uint32_t cell_key(int cx, int cy, int cz) {
    return spread3((uint32_t)cx) | (spread3((uint32_t)cy) << 1) | (spread3((uint32_t)cz) << 2);
}
__device__ __forceinline__ uint32_t cell_of(float x, float y, float z, int K) {
    return cell_key(cell_coord(x, K), cell_coord(y, K), cell_coord(z, K));
}

// Count the elements of each cell. POST = false: the live dense slots (the
// heap's state before the update); POST = true: the sorted positions below
// n_live (the updated positions).
template <bool POST>
__global__ void k_cell_count(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbWs ws) {
    const uint32_t n = POST ? n_bodies(ws) : n_dense(H);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        uint32_t c;
        if (POST) {
            const float4 u = ws.npos[e];
            c = cell_of(u.x, u.y, u.z, ws.K);
        } else {
            if (!slot_live(H, e)) continue;
            const dsr_ref r = slot_ref(H, e);
            c = cell_of(*fld(H, r, PX), *fld(H, r, PY), *fld(H, r, PZ), ws.K);
        }
        ws.ckey[e] = c;
        atomicAdd(ws.ccount + c, 1u);
    }
}

// Exclusive prefix sum of the cell counts, in two launches of NKEYS / 1024
// CTAs: each CTA sums its 1024 cells (k_cell_sum), then each CTA scans its
// cells from the sum of the CTAs before it (k_cell_scan). For the first order
// the total is the live body count, and the step's near-pair count starts
// at 0.
constexpr uint32_t SCAN_CTAS = NKEYS / 1024;

__global__ void __launch_bounds__(1024) k_cell_sum(const __grid_constant__ NbWs ws) {
    const uint32_t v = __reduce_add_sync(0xFFFFFFFFu, ws.ccount[blockIdx.x * 1024 + threadIdx.x]);
    __shared__ uint32_t w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        const uint32_t t = __reduce_add_sync(0xFFFFFFFFu, w[threadIdx.x]);
        if (threadIdx.x == 0) ws.csum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) k_cell_scan(const __grid_constant__ NbWs ws, int post) {
    __shared__ uint32_t w[32];
    __shared__ uint32_t base;
    uint32_t* coff = post ? ws.coff2 : ws.coff;
    if (threadIdx.x < 32) {
        uint32_t b = 0;
        for (uint32_t k = threadIdx.x; k < blockIdx.x; k += 32) b += ws.csum[k];
        b = __reduce_add_sync(0xFFFFFFFFu, b);
        if (threadIdx.x == 0) base = b;
    }
    const uint32_t c = blockIdx.x * 1024 + threadIdx.x;
    const uint32_t v = ws.ccount[c];
    const unsigned lane = threadIdx.x & 31;
    uint32_t x = v;  // inclusive warp scan
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) w[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t t = w[threadIdx.x];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (threadIdx.x >= (unsigned)o) t += y;
        }
        w[threadIdx.x] = t;  // inclusive scan of the warp totals
    }
    __syncthreads();
    const uint32_t before = base + (threadIdx.x >= 32 ? w[(threadIdx.x >> 5) - 1] : 0u) + x - v;
    coff[c] = before;
    if (c == NKEYS - 1) {
        coff[NKEYS] = before + v;
        if (!post) {
            *ws.n_live = before + v;
            *ws.npairs = 0;
        }
    }
}

// Place every counted element in its cell's range (in arbitrary order within
// the cell); the counts return to zero.
template <bool POST>
__global__ void k_cell_place(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbWs ws) {
    const uint32_t n = POST ? n_bodies(ws) : n_dense(H);
    const uint32_t* coff = POST ? ws.coff2 : ws.coff;
    uint32_t* out = POST ? ws.perm2 : ws.perm;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        if (!POST && !slot_live(H, e)) continue;
        const uint32_t c = ws.ckey[e];
        out[coff[c] + atomicSub(ws.ccount + c, 1u) - 1u] = e;
    }
}

// Id of a placed element: of the body in dense slot e, or at sorted position e.
template <bool POST>
__device__ __forceinline__ int32_t elem_id(const dsr_dev_heap& H, const NbWs& ws, uint32_t e) {
    return POST ? ws.id[e] : *dsr_field<int32_t>(H, BODY, slot_ref(H, e), ID);
}

// The elements of each cell in order of body id (ids are unique): one thread
// per cell, insertion sort.
template <bool POST>
__global__ void k_cell_order(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbWs ws) {
    const uint32_t* coff = POST ? ws.coff2 : ws.coff;
    uint32_t* seg = POST ? ws.perm2 : ws.perm;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < NKEYS; c += gridDim.x * blockDim.x) {
        const uint32_t a = coff[c], b = coff[c + 1];
        for (uint32_t u = a + 1; u < b; ++u) {
            const uint32_t x = seg[u];
            const int32_t key = elem_id<POST>(H, ws, x);
            uint32_t v = u;
            while (v > a && elem_id<POST>(H, ws, seg[v - 1]) > key) {
                seg[v] = seg[v - 1];
                --v;
            }
            seg[v] = x;
        }
    }
}

// Sorted positions: one CTA per tile of 256. Each position gets its body's
// state (or an empty entry past the live bodies), each tile the bounding box
// of its bodies' high-word positions (empty: low corner +FLT_MAX).
__global__ void __launch_bounds__(TILE) k_gather(const __grid_constant__ dsr_dev_heap H,
                                                 const __grid_constant__ NbWs ws) {
    __shared__ float red[6][TILE / 32];
    const uint32_t nl = n_bodies(ws), np = n_padded(ws);
    for (uint32_t t = blockIdx.x; t * TILE < np; t += gridDim.x) {
        const uint32_t p = t * TILE + threadIdx.x;
        float b[6] = {FLT_MAX, FLT_MAX, FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX};
        if (p < nl) {
            const dsr_ref r = slot_ref(H, ws.perm[p]);
            const float4 u = make_float4(*fld(H, r, PX), *fld(H, r, PY), *fld(H, r, PZ), *fld(H, r, MASS));
            ws.pos[p] = u;
            ws.pd[p] = d4(get2(H, r, PX), get2(H, r, PY), get2(H, r, PZ), get2(H, r, MASS));
            ws.id[p] = *dsr_field<int32_t>(H, BODY, r, ID);
            ws.sref[p] = r;
            b[0] = b[3] = u.x, b[1] = b[4] = u.y, b[2] = b[5] = u.z;
        } else {
            ws.pos[p] = make_float4(0.f, 0.f, 0.f, 0.f);
            ws.pd[p] = d4(0.0, 0.0, 0.0, 0.0);
            ws.id[p] = 0x7FFFFFFF;
            ws.sref[p] = DSR_NULL;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const float v = __shfl_xor_sync(0xFFFFFFFFu, b[k], o);
                b[k] = k < 3 ? fminf(b[k], v) : fmaxf(b[k], v);
            }
        }
        __syncthreads();  // the previous tile's reduction has been read
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int k = 0; k < 6; ++k) red[k][threadIdx.x >> 5] = b[k];
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int w = 1; w < TILE / 32; ++w)
#pragma unroll
                for (int k = 0; k < 6; ++k) b[k] = k < 3 ? fminf(b[k], red[k][w]) : fmaxf(b[k], red[k][w]);
            ws.tbox[2 * t] = make_float4(b[0], b[1], b[2], 0.f);
            ws.tbox[2 * t + 1] = make_float4(b[3], b[4], b[5], 0.f);
        }
    }
}

// True unless every pair between the boxes [la, ha] and [lb, hb] is at least
// r_near apart, with room for the rounding of the FP32 r^2 (the near test
// then fails for all of them). Empty boxes are far from everything.
__device__ __forceinline__ bool boxes_near(float4 la, float4 ha, float4 lb, float4 hb, float rn2) {
    if (!(rn2 > 0.f) || la.x > ha.x || lb.x > hb.x) return false;
    const float dx = fmaxf(0.f, fmaxf(lb.x - ha.x, la.x - hb.x));
    const float dy = fmaxf(0.f, fmaxf(lb.y - ha.y, la.y - hb.y));
    const float dz = fmaxf(0.f, fmaxf(lb.z - ha.z, la.z - hb.z));
    return !(dx * dx + dy * dy + dz * dz >= rn2 * 1.0001f);
}

// 1/sqrt(x) by the PTX approximate reciprocal square root with subnormal
// inputs flushed to zero; used only where x >= eps^2 >= FLT_MIN (or +inf, for
// an excluded pair), so the flush never applies.
__device__ __forceinline__ float rsqrt_normal(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float f_inf() { return __int_as_float(0x7F800000); }

// The FP32 pair test shared by the force kernels and the near field: the
// near field takes exactly the pairs the force kernels leave out.
__device__ __forceinline__ float pair_r2(float4 pj, float px, float py, float pz, float eps2, float& dx, float& dy,
                                         float& dz) {
    dx = pj.x - px, dy = pj.y - py, dz = pj.z - pz;
    return fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
}

// ---------------------------------------------------------------------------
// FP32 pair forces
// ---------------------------------------------------------------------------
// Split form. A row item is ROW = TILE * RB sorted positions (RB per thread:
// position row * ROW + k * TILE + threadIdx.x), the j tiles are cut into
// `ns` slices, and a work item is one (row item, slice) pair; `ns` follows
// from the padded count on the device (n_slices), so the items fill about
// `grid` CTAs whatever the live count. Each item writes its partial sums to
// part[slice][p]; the update reads the slices back in slice order.
//
// Register blocking. Every lane of a warp reads the same j body from shared
// memory (a broadcast); with RB bodies per thread each load feeds RB pairs.
//
// Near tiles. A tile whose bounding box comes within r_near of the row's
// runs the excluding loop: a pair closer than r_near (the same FP32 r^2 the
// near field tests) gets r^2 = +inf, so rsqrt gives 0 and the pair adds
// nothing. Other tiles run the plain loop. In spatial order few tiles are
// near a row, and the choice is uniform across the CTA.
__device__ __forceinline__ uint32_t n_slices(uint32_t nr, uint32_t nj, uint32_t grid) {
    if (!nr) return 0;
    const uint32_t k = grid / nr;
    return k < 1 ? 1 : (k > nj ? nj : k);
}

struct SplitShape {
    uint32_t n, nj, nr, ns;  // padded count, j tiles, row items, slices
};

__device__ __forceinline__ SplitShape split_shape(const NbWs& ws, uint32_t grid, int rb) {
    SplitShape q;
    q.n = n_padded(ws);
    q.nj = q.n / TILE;
    q.nr = q.n / (TILE * rb);
    q.ns = n_slices(q.nr, q.nj, grid);
    return q;
}

// One tile of j bodies for the thread's RB bodies, in chunks of CHUNK
// pairs: a chunk is summed in FP32 and added to (a, c) with Kahan
// compensation. In spatial order a tile's terms for a body point much the
// same way, so a plain 256-term FP32 sum would round at the size of the
// whole tile's pull; chunks bound that rounding to the size of 32 terms.
constexpr int CHUNK = 32;

template <bool SOFT, bool EXCLUDE>
__device__ __forceinline__ void force_tile(const float4* sp, const float* px, const float* py, const float* pz,
                                           float eps2, float rn2, float* ax, float* ay, float* az, float* cx,
                                           float* cy, float* cz) {
    for (int j0 = 0; j0 < TILE; j0 += CHUNK) {
        float tx[RB], ty[RB], tz[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) tx[k] = ty[k] = tz[k] = 0.f;
#pragma unroll 4
        for (int j = j0; j < j0 + CHUNK; ++j) {
            const float4 pj = sp[j];
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                float dx, dy, dz;
                float r2 = pair_r2(pj, px[k], py[k], pz[k], eps2, dx, dy, dz);
                if (EXCLUDE) r2 = r2 < rn2 ? f_inf() : r2;
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
}

template <bool SOFT>
__global__ void __launch_bounds__(TILE) k_force_part(const __grid_constant__ dsr_dev_heap H,
                                                     const __grid_constant__ NbArgs a) {
    (void)H;
    __shared__ float4 sp[TILE];
    const SplitShape q = split_shape(a.ws, gridDim.x, RB);
    const float eps2 = (float)(a.p.eps * a.p.eps);
    const float rn2 = (float)(a.p.r_near * a.p.r_near);
    for (uint32_t item = blockIdx.x; item < q.nr * q.ns; item += gridDim.x) {
        const uint32_t row = item % q.nr, sl = item / q.nr;
        const uint32_t g0 = row * ROW + threadIdx.x;
        float4 rlo = a.ws.tbox[2 * RB * row], rhi = a.ws.tbox[2 * RB * row + 1];
#pragma unroll
        for (int k = 1; k < RB; ++k) {
            const float4 l = a.ws.tbox[2 * (RB * row + k)], h = a.ws.tbox[2 * (RB * row + k) + 1];
            rlo = make_float4(fminf(rlo.x, l.x), fminf(rlo.y, l.y), fminf(rlo.z, l.z), 0.f);
            rhi = make_float4(fmaxf(rhi.x, h.x), fmaxf(rhi.y, h.y), fmaxf(rhi.z, h.z), 0.f);
        }
        float px[RB], py[RB], pz[RB];
        float ax[RB], ay[RB], az[RB], cx[RB], cy[RB], cz[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            const float4 u = a.ws.pos[g0 + k * TILE];
            px[k] = u.x, py[k] = u.y, pz[k] = u.z;
            ax[k] = ay[k] = az[k] = cx[k] = cy[k] = cz[k] = 0.f;
        }
        for (uint32_t t = q.nj * sl / q.ns; t < q.nj * (sl + 1) / q.ns; ++t) {
            __syncthreads();
            sp[threadIdx.x] = a.ws.pos[t * TILE + threadIdx.x];
            __syncthreads();
            if (boxes_near(rlo, rhi, a.ws.tbox[2 * t], a.ws.tbox[2 * t + 1], rn2))
                force_tile<SOFT, true>(sp, px, py, pz, eps2, rn2, ax, ay, az, cx, cy, cz);
            else
                force_tile<SOFT, false>(sp, px, py, pz, eps2, rn2, ax, ay, az, cx, cy, cz);
        }
        float4* out = a.ws.part + (size_t)sl * q.n;
#pragma unroll
        for (int k = 0; k < RB; ++k) out[g0 + k * TILE] = make_float4(ax[k], ay[k], az[k], 0.f);
    }
}

// Unsplit form (the allocation-free step): one thread per sorted position,
// one CTA per tile of positions; the same pair test, exclusion and term.
__global__ void __launch_bounds__(TILE) k_force(const __grid_constant__ dsr_dev_heap H,
                                                const __grid_constant__ NbArgs a) {
    (void)H;
    __shared__ float4 sp[TILE];
    const uint32_t n = n_padded(a.ws);
    const uint32_t base = blockIdx.x * TILE;
    if (base >= n) return;
    const uint32_t g = base + threadIdx.x;
    const float4 pi = a.ws.pos[g];
    const float4 rlo = a.ws.tbox[2 * blockIdx.x], rhi = a.ws.tbox[2 * blockIdx.x + 1];
    const float eps2 = (float)(a.p.eps * a.p.eps);
    const float rn2 = (float)(a.p.r_near * a.p.r_near);
    float ax = 0.f, ay = 0.f, az = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    for (uint32_t t0 = 0; t0 < n; t0 += TILE) {
        __syncthreads();
        sp[threadIdx.x] = a.ws.pos[t0 + threadIdx.x];
        __syncthreads();
        const bool near = boxes_near(rlo, rhi, a.ws.tbox[2 * (t0 / TILE)], a.ws.tbox[2 * (t0 / TILE) + 1], rn2);
        for (int j0 = 0; j0 < TILE; j0 += CHUNK) {
            float tx = 0.f, ty = 0.f, tz = 0.f;
            for (int j = j0; j < j0 + CHUNK; ++j) {
                float dx, dy, dz;
                float r2 = pair_r2(sp[j], pi.x, pi.y, pi.z, eps2, dx, dy, dz);
                if (near && r2 < rn2) r2 = f_inf();
                const float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                const float w = sp[j].w * inv * inv * inv;
                tx = fmaf(w, dx, tx);
                ty = fmaf(w, dy, ty);
                tz = fmaf(w, dz, tz);
            }
            kahan_add(ax, cx, tx);
            kahan_add(ay, cy, ty);
            kahan_add(az, cz, tz);
        }
    }
    a.ws.part[g] = make_float4(ax, ay, az, 0.f);
}

// ---------------------------------------------------------------------------
// FP64 pair forces
// ---------------------------------------------------------------------------
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

// Split form, RB64 positions per thread, every pair in FP64.
__global__ void __launch_bounds__(TILE) k_force_part64(const __grid_constant__ dsr_dev_heap H,
                                                       const __grid_constant__ NbArgs a) {
    (void)H;
    __shared__ D4 sp[TILE];
    const SplitShape q = split_shape(a.ws, gridDim.x, RB64);
    const double eps2 = a.p.eps * a.p.eps;
    for (uint32_t item = blockIdx.x; item < q.nr * q.ns; item += gridDim.x) {
        const uint32_t row = item % q.nr, sl = item / q.nr;
        const uint32_t g0 = row * TILE * RB64 + threadIdx.x;
        double px[RB64], py[RB64], pz[RB64], ax[RB64], ay[RB64], az[RB64];
#pragma unroll
        for (int k = 0; k < RB64; ++k) {
            const D4 u = a.ws.pd[g0 + k * TILE];
            px[k] = u.x, py[k] = u.y, pz[k] = u.z;
            ax[k] = ay[k] = az[k] = 0.0;
        }
        for (uint32_t t = q.nj * sl / q.ns; t < q.nj * (sl + 1) / q.ns; ++t) {
            __syncthreads();
            sp[threadIdx.x] = a.ws.pd[t * TILE + threadIdx.x];
            __syncthreads();
#pragma unroll 2
            for (int j = 0; j < TILE; ++j) {
                const D4 pj = sp[j];
#pragma unroll
                for (int k = 0; k < RB64; ++k) pair64(pj, px[k], py[k], pz[k], eps2, ax[k], ay[k], az[k]);
            }
        }
        D4* out = a.ws.part64 + (size_t)sl * q.n;
#pragma unroll
        for (int k = 0; k < RB64; ++k) out[g0 + k * TILE] = d4(ax[k], ay[k], az[k], 0.0);
    }
}

// Unsplit form (the allocation-free step).
__global__ void __launch_bounds__(TILE) k_force64(const __grid_constant__ dsr_dev_heap H,
                                                  const __grid_constant__ NbArgs a) {
    (void)H;
    __shared__ D4 sp[TILE];
    const uint32_t n = n_padded(a.ws);
    const uint32_t base = blockIdx.x * TILE;
    if (base >= n) return;
    const uint32_t g = base + threadIdx.x;
    const D4 pi = a.ws.pd[g];
    const double eps2 = a.p.eps * a.p.eps;
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (uint32_t t0 = 0; t0 < n; t0 += TILE) {
        __syncthreads();
        sp[threadIdx.x] = a.ws.pd[t0 + threadIdx.x];
        __syncthreads();
        for (int j = 0; j < TILE; ++j) pair64(sp[j], pi.x, pi.y, pi.z, eps2, ax, ay, az);
    }
    a.ws.part64[g] = d4(ax, ay, az, 0.0);
}

// ---------------------------------------------------------------------------
// update, partner search, merge
// ---------------------------------------------------------------------------
// Visit the sorted entries of the cells around (and including) the cell of
// (x, y, z) that lie within `rad` of the point on each axis (of the 27
// neighbours, those the search radius reaches), cells in a fixed order:
// fn(q) for each position q of the first order, or (POST) for the position
// perm2[q] of each entry q of the second order. Cells are at least as wide
// as rad, so no other cell holds a body within rad.
// The same walk restricted to the cells of column ix - 1 + slab (slab 0, 1
// or 2: the lower, own and upper x neighbour), nothing when the search does
// not reach that column.
template <class F>
__device__ __forceinline__ void for_neighbours_slab(const NbWs& ws, float x, float y, float z, float rad, int slab,
                                                    F fn) {
    const int K = ws.K;
    const float inv = 1.f / (float)K;
    const int cx = cell_coord(x, K), cy = cell_coord(y, K), cz = cell_coord(z, K);
    const int ix = cx - 1 + slab;
    if (slab == 0 && !(cx > 0 && x - (float)cx * inv < rad)) return;
    if (slab == 2 && !(cx < K - 1 && (float)(cx + 1) * inv - x < rad)) return;
    const int y0 = cy > 0 && y - (float)cy * inv < rad ? cy - 1 : cy;
    const int y1 = cy < K - 1 && (float)(cy + 1) * inv - y < rad ? cy + 1 : cy;
    const int z0 = cz > 0 && z - (float)cz * inv < rad ? cz - 1 : cz;
    const int z1 = cz < K - 1 && (float)(cz + 1) * inv - z < rad ? cz + 1 : cz;
    for (int iy = y0; iy <= y1; ++iy)
        for (int iz = z0; iz <= z1; ++iz) {
            const uint32_t c = cell_key(ix, iy, iz);
            for (uint32_t q = ws.coff[c]; q < ws.coff[c + 1]; ++q) fn(q);
        }
}

template <bool POST, class F>
__device__ __forceinline__ void for_neighbours(const NbWs& ws, float x, float y, float z, float rad, F fn) {
    const int K = ws.K;
    const float inv = 1.f / (float)K;
    const int cx = cell_coord(x, K), cy = cell_coord(y, K), cz = cell_coord(z, K);
    // a neighbour below (above) on an axis is needed when the point is within
    // rad of that face of its cell; border cells extend to infinity
    const int x0 = cx > 0 && x - (float)cx * inv < rad ? cx - 1 : cx;
    const int x1 = cx < K - 1 && (float)(cx + 1) * inv - x < rad ? cx + 1 : cx;
    const int y0 = cy > 0 && y - (float)cy * inv < rad ? cy - 1 : cy;
    const int y1 = cy < K - 1 && (float)(cy + 1) * inv - y < rad ? cy + 1 : cy;
    const int z0 = cz > 0 && z - (float)cz * inv < rad ? cz - 1 : cz;
    const int z1 = cz < K - 1 && (float)(cz + 1) * inv - z < rad ? cz + 1 : cz;
    const uint32_t* coff = POST ? ws.coff2 : ws.coff;
    for (int ix = x0; ix <= x1; ++ix)
        for (int iy = y0; iy <= y1; ++iy)
            for (int iz = z0; iz <= z1; ++iz) {
                const uint32_t c = cell_key(ix, iy, iz);
                for (uint32_t q = coff[c]; q < coff[c + 1]; ++q) fn(POST ? ws.perm2[q] : q);
            }
}

// r^-3 for r2 = r^2 in FP64. Newton's iteration for 1/sqrt(r2), y <- y (3 -
// r2 y^2) / 2, from the FP32 estimate: a relative error e becomes about
// 1.5 e^2, so two steps take the estimate's 2^-22 below FP64 rounding, with
// six FP64 multiply-adds where a square root and a division cost several
// times that on GB300's FP64 units. Outside the FP32 range of the estimate
// the plain expression is used.
__device__ __forceinline__ double rsqrt_cubed(double r2) {
    if (!(r2 >= (double)FLT_MIN && r2 <= (double)FLT_MAX)) return 1.0 / (r2 * sqrt(r2));
    double y = (double)rsqrtf((float)r2);
    y = y * (1.5 - 0.5 * r2 * y * y);
    y = y * (1.5 - 0.5 * r2 * y * y);
    return y * y * y;
}

// Far field of the body at sorted position p: its slices summed in slice
// order. FP32 slices are summed as FP32 pairs (error-free additions), which
// is as exact here as FP64 additions and keeps the FP64 units, a small
// fraction of GB300's FP32 rate, free for the near field and the update.
__device__ __forceinline__ void far_field(const NbArgs& a, uint32_t p, uint32_t ns, size_t stride, bool f64,
                                          double& ax, double& ay, double& az) {
    if (f64) {
        for (uint32_t k = 0; k < ns; ++k) {
            const D4 v = a.ws.part64[k * stride + p];
            ax += v.x;
            ay += v.y;
            az += v.z;
        }
        return;
    }
    float sx = 0.f, sy = 0.f, sz = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;
    // slices loaded four at a time, then added in order
    uint32_t k = 0;
    for (; k + 4 <= ns; k += 4) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = a.ws.part[(k + u) * stride + p];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            two_sum_add(sx, ex, v[u].x);
            two_sum_add(sy, ey, v[u].y);
            two_sum_add(sz, ez, v[u].z);
        }
    }
    for (; k < ns; ++k) {
        const float4 v = a.ws.part[k * stride + p];
        two_sum_add(sx, ex, v.x);
        two_sum_add(sy, ey, v.y);
        two_sum_add(sz, ez, v.z);
    }
    ax = (double)sx + (double)ex;
    ay = (double)sy + (double)ey;
    az = (double)sz + (double)ez;
}

// One near pair in FP64 from the full state: the acceleration of the body
// at full position pi from body j (position and mass pj).
__device__ __forceinline__ void near_term(const D4& pi, const D4& pj, double eps2d, double& cx, double& cy,
                                          double& cz) {
    const double ex = pj.x - pi.x, ey = pj.y - pi.y, ez = pj.z - pi.z;
    const double w = pj.w * rsqrt_cubed(ex * ex + ey * ey + ez * ez + eps2d);
    cx = w * ex;
    cy = w * ey;
    cz = w * ez;
}

// A queued near pair of a warp and its FP64 term.
struct NearSlot {
    uint32_t p, q;
    double x, y, z;
};
constexpr int NEAR_Q = 4;                       // pairs a lane queues; more are computed in place
constexpr int NEAR_SLOTS = 32 * NEAR_Q;         // per warp
constexpr int UPDATE_THREADS = 256;

// The update: four lanes per body. Lanes 0-2 of a body's quad take the near
// field (FP32 pairs only) from the lower, own and upper x column of cells
// around it: the pairs the force kernels left out (the same FP32 test),
// added in FP64 from the full state in cell and body order. Lane 3 sums the
// far-field slices. Lane k of the quad (k < 3) then adds the four parts of
// axis k in a fixed order (far, then the columns from low to high), so a
// step stays deterministic, and does that axis of v += a dt, x += v dt
// (semi-implicit Euler) in FP64 on the full state, stored back as FP32
// pairs; lane 3 writes the mass parts of the new state. `grid` is the split
// force kernel's grid (0: the unsplit kernel's single slice).
//
// FP64 work in a warp. GB300 issues FP64 instructions at a small fraction of
// its FP32 rate, and a warp instruction costs the same however few lanes it
// runs for. A near pair found by one lane in a divergent branch would cost
// its ~20 FP64 instructions for the whole warp. So the walk only queues the
// pairs (up to NEAR_Q a lane, in walk order) in a per-warp list, compacted
// by a prefix sum; the warp then computes the list's terms with all lanes
// busy, and each lane adds its own terms back in walk order. A lane with more
// than NEAR_Q pairs computes the rest in place, in order, into a second sum.
// For the same reason the update is split by axis over the quad.
// At least three CTAs per SM (at most 85 registers): the walk is a chain of
// dependent loads, and with two (90 registers unbounded) it waited on them;
// four spilled and made the step slower.
constexpr int UPDATE_MIN_CTAS = 3;
__global__ void __launch_bounds__(UPDATE_THREADS, UPDATE_MIN_CTAS) k_update(const __grid_constant__ dsr_dev_heap H,
                                                           const __grid_constant__ NbArgs a, uint32_t grid) {
    __shared__ NearSlot slots[UPDATE_THREADS / 32][NEAR_SLOTS];
    const bool f64 = a.p.pair_precision == DSR_NBODY_PAIRS_FP64;
    uint32_t ns = 1;
    size_t stride = 0;
    if (grid) {
        const SplitShape q = split_shape(a.ws, grid, f64 ? RB64 : RB);
        ns = q.ns;
        stride = q.n;
    }
    const uint32_t n = n_bodies(a.ws);
    const unsigned lane = threadIdx.x & 31u, sub = lane & 3u, quad = lane & ~3u;
    NearSlot* sl = slots[threadIdx.x >> 5];
    const float rn2 = (float)(a.p.r_near * a.p.r_near);
    const float rad = (float)(a.p.r_near * 1.001);
    const float eps2 = (float)(a.p.eps * a.p.eps);
    const double eps2d = a.p.eps * a.p.eps;
    const bool near_on = !f64 && rn2 > 0.f;
    uint32_t near = 0;
    // 4 n lanes, rounded up to whole warps: every lane of a warp runs the
    // same iterations, so the warp-wide steps below see the whole warp
    const uint64_t lanes = ((uint64_t)n * 4 + 31) & ~31ull;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < lanes; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t p = (uint32_t)(t >> 2);
        const bool live = p < n;
        double ax = 0.0, ay = 0.0, az = 0.0;  // far field (lane 3) or queued near terms (lanes 0-2)
        double ox = 0.0, oy = 0.0, oz = 0.0;  // near terms beyond the queue
        uint32_t cnt = 0, qd[NEAR_Q] = {0, 0, 0, 0};
        if (live && sub == 3) {
            far_field(a, p, ns, stride, f64, ax, ay, az);
        } else if (live && near_on) {
            const D4 pi = a.ws.pd[p];
            const float4 u = a.ws.pos[p];
            // pairs the FP32 test can pass lie within r_near of the body, up
            // to the rounding of r^2 (a margin of 1e-3 relative covers it)
            for_neighbours_slab(a.ws, u.x, u.y, u.z, rad, (int)sub, [&](uint32_t q) {
                if (q == p) return;
                float dx, dy, dz;
                if (!(pair_r2(a.ws.pos[q], u.x, u.y, u.z, eps2, dx, dy, dz) < rn2)) return;
                if (cnt < NEAR_Q) {
#pragma unroll
                    for (int e = 0; e < NEAR_Q; ++e)
                        if ((int)cnt == e) qd[e] = q;
                } else {
                    double cx, cy, cz;
                    near_term(pi, a.ws.pd[q], eps2d, cx, cy, cz);
                    ox += cx;
                    oy += cy;
                    oz += cz;
                }
                ++cnt;
            });
        }
        near += cnt;
        // compact the queued pairs of the warp: exclusive prefix sum of m
        const uint32_t m = cnt < NEAR_Q ? cnt : NEAR_Q;
        uint32_t incl = m;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if ((int)lane >= o) incl += v;
        }
        const uint32_t excl = incl - m, total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        if (total) {
#pragma unroll
            for (int e = 0; e < NEAR_Q; ++e)
                if ((uint32_t)e < m) sl[excl + e].p = p, sl[excl + e].q = qd[e];
            __syncwarp();
            for (uint32_t k = lane; k < total; k += 32) {
                double cx, cy, cz;
                near_term(a.ws.pd[sl[k].p], a.ws.pd[sl[k].q], eps2d, cx, cy, cz);
                sl[k].x = cx, sl[k].y = cy, sl[k].z = cz;
            }
            __syncwarp();
#pragma unroll
            for (int e = 0; e < NEAR_Q; ++e)
                if ((uint32_t)e < m) ax += sl[excl + e].x, ay += sl[excl + e].y, az += sl[excl + e].z;
            __syncwarp();  // the list is read before the next iteration writes it
        }
        if (cnt > NEAR_Q) ax += ox, ay += oy, az += oz;
        // lane k of the quad gathers axis k: far (lane 3), then columns 0, 1, 2
        double part[4];
#pragma unroll
        for (int src = 0; src < 4; ++src) {
            const double vx = __shfl_sync(0xFFFFFFFFu, ax, quad + src);
            const double vy = __shfl_sync(0xFFFFFFFFu, ay, quad + src);
            const double vz = __shfl_sync(0xFFFFFFFFu, az, quad + src);
            part[src] = sub == 0 ? vx : (sub == 1 ? vy : vz);
        }
        if (!live) continue;
        const dsr_ref r = a.ws.sref[p];
        double* npd = reinterpret_cast<double*>(a.ws.npd + p);
        double* nvd = reinterpret_cast<double*>(a.ws.nvd + p);
        float* npos = reinterpret_cast<float*>(a.ws.npos + p);
        if (sub < 3) {
            const double g = ((part[3] + part[0]) + part[1]) + part[2];
            const double x0 = reinterpret_cast<const double*>(a.ws.pd + p)[sub];
            const double v = get2(H, r, VX + (int)sub) + a.p.G * g * a.p.dt;
            const double x = x0 + v * a.p.dt;
            put2(H, r, VX + (int)sub, v);
            put2(H, r, PX + (int)sub, x);
            npos[sub] = *fld(H, r, PX + (int)sub);
            npd[sub] = x;
            nvd[sub] = v;
        } else {
            npos[3] = *fld(H, r, MASS);
            npd[3] = a.ws.pd[p].w;
            nvd[3] = 0.0;
        }
    }
    near = __reduce_add_sync(0xFFFFFFFFu, near);
    if ((threadIdx.x & 31) == 0 && near) atomicAdd(a.ws.npairs, near);
}

// FP32 radius that selects merge candidates: r_merge plus a margin above the
// rounding of the high words (positions of magnitude below 64).
__device__ __forceinline__ float wide_merge2(const NbArgs& a) {
    const float rw = (float)(a.p.r_merge * (1.0 + 1e-3) + 1e-5);
    return rw * rw;
}

// Partner of the body at sorted position p, on the updated positions: the
// lowest id within r_merge (the FP32 test on the high words, widened, picks
// candidates from the 27 cells around its new cell; the FP64 distance of the
// full positions decides).
__global__ void k_partner(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbArgs a) {
    (void)H;
    const uint32_t n = n_bodies(a.ws);
    const float rw2 = wide_merge2(a);
    const double rm2 = a.p.r_merge * a.p.r_merge;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float4 u = a.ws.npos[p];
        const D4 ud = a.ws.npd[p];
        int32_t best_id = 0x7FFFFFFF, best = -1;
        for_neighbours<true>(a.ws, u.x, u.y, u.z, sqrtf(rw2) * 1.001f, [&](uint32_t q) {
            if (q == p) return;
            const float4 v = a.ws.npos[q];
            const float dx = v.x - u.x, dy = v.y - u.y, dz = v.z - u.z;
            if (!(fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rw2)) return;
            const int32_t jid = a.ws.id[q];
            if (jid >= best_id) return;
            const D4 vd = a.ws.npd[q];
            const double ex = vd.x - ud.x, ey = vd.y - ud.y, ez = vd.z - ud.z;
            if (ex * ex + ey * ey + ez * ez < rm2) {
                best_id = jid;
                best = (int32_t)q;
            }
        });
        a.ws.partner[p] = best;
    }
}

// Merge mutual partners in FP64; the higher id deletes itself. Last kernel
// of the step: its last CTA resets R and advances the step counter.
__global__ void k_merge(const __grid_constant__ dsr_dev_heap H, const __grid_constant__ NbArgs a) {
    const uint32_t n = n_bodies(a.ws);
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t p = base + threadIdx.x;
        if (p >= n) continue;
        const int32_t j = a.ws.partner[p];
        if (j < 0 || a.ws.partner[j] != (int32_t)p) continue;
        const dsr_ref r = a.ws.sref[p];
        if (a.ws.id[p] > a.ws.id[j]) {
            dsr_delete(H, r);
            continue;
        }
        const D4 pg = a.ws.npd[p], pj = a.ws.npd[j];
        const D4 vg = a.ws.nvd[p], vj = a.ws.nvd[j];
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
            a.ws.log[3 * k + 1] = a.ws.id[p];
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
    return p && p->dt > 0.0 && p->eps >= 0.0 && p->r_merge >= 0.0 && p->r_near >= 0.0 && p->r_near < 1.0 &&
           p->r_merge < 1.0 && (p->pair_precision == DSR_NBODY_PAIRS_FP32 || p->pair_precision == DSR_NBODY_PAIRS_FP64);
}

// Cells per axis: as many as fit, up to KMAX, with cells at least as wide as
// the near radius and the widened merge radius (then the pairs either test
// selects lie in adjacent cells).
int cells_per_axis(const dsr_nbody_params& p) {
    const double rw = p.r_merge * (1.0 + 1e-3) + 1e-5;
    const double r = (p.r_near > rw ? p.r_near : rw) * 1.001;
    const int K = (int)(1.0 / r);
    return K < 1 ? 1 : (K > KMAX ? KMAX : K);
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Grid of a split all-pairs kernel: four waves of its resident CTAs.
uint32_t split_grid(const dsr_heap* h, const void* kernel) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, TILE, 0) != cudaSuccess || occ < 1) occ = 1;
    return (uint32_t)(4 * occ * h->sm_count);
}

struct SplitGrids {
    uint32_t force, force64;
};

SplitGrids split_grids(const dsr_heap* h) {
    return {split_grid(h, (const void*)k_force_part<true>), split_grid(h, (const void*)k_force_part64)};
}

// Padded positions for a heap of S slots.
uint64_t padded(uint64_t S) { return (S + ROW - 1) / ROW * ROW; }

// Slice entries of a split kernel over at most P padded positions: at most
// max(grid / rows, 1) slices (and no more than the j tiles) of P entries.
size_t slots_for(uint64_t P, uint32_t grid, int rb) {
    const uint64_t nr = P / (TILE * rb);
    uint64_t ns = nr ? grid / nr : 1;
    if (ns < 1) ns = 1;
    if (ns > P / TILE) ns = P / TILE;
    return (size_t)ns * P;
}
// Bytes of the force slice buffer: FP32 sums (16 bytes an entry) or FP64 sums
// (32 bytes), whichever needs more. (A step with fewer live bodies has fewer
// rows, more slices and a smaller padded count; ns * n stays within this.)
size_t part_bytes(uint64_t P, SplitGrids g) {
    size_t m = 0;
    for (uint64_t n = ROW; n <= P; n += ROW) {  // every padded count a step can have
        const size_t a = slots_for(n, g.force, RB) * 16, b = slots_for(n, g.force64, RB64) * 32;
        if (a > m) m = a;
        if (b > m) m = b;
    }
    return m;
}

// The spatial-order and per-position arrays of P padded positions, carved
// from p (advanced).
void carve_common(uint8_t*& p, uint64_t P, NbWs& w) {
    w.ccount = reinterpret_cast<uint32_t*>(p);
    p += round256(NKEYS * 4);
    w.coff = reinterpret_cast<uint32_t*>(p);
    p += round256((NKEYS + 1) * 4);
    w.coff2 = reinterpret_cast<uint32_t*>(p);
    p += round256((NKEYS + 1) * 4);
    w.csum = reinterpret_cast<uint32_t*>(p);
    p += 256;
    w.ckey = reinterpret_cast<uint32_t*>(p);
    p += round256(P * 4);
    w.perm = reinterpret_cast<uint32_t*>(p);
    p += round256(P * 4);
    w.perm2 = reinterpret_cast<uint32_t*>(p);
    p += round256(P * 4);
    w.pos = reinterpret_cast<float4*>(p);
    p += round256(P * 16);
    w.pd = reinterpret_cast<D4*>(p);
    p += round256(P * 32);
    w.id = reinterpret_cast<int32_t*>(p);
    p += round256(P * 4);
    w.sref = reinterpret_cast<dsr_u64*>(p);
    p += round256(P * 8);
    w.tbox = reinterpret_cast<float4*>(p);
    p += round256(P / TILE * 32);
    w.npos = reinterpret_cast<float4*>(p);
    p += round256(P * 16);
    w.npd = reinterpret_cast<D4*>(p);
    p += round256(P * 32);
    w.nvd = reinterpret_cast<D4*>(p);
    p += round256(P * 32);
    w.partner = reinterpret_cast<int32_t*>(p);
    p += round256(P * 4);
}
size_t common_bytes(uint64_t P) {
    return round256(NKEYS * 4) + 2 * round256((NKEYS + 1) * 4) + 256 + 3 * round256(P * 4) + round256(P * 16) +
           round256(P * 32) + round256(P * 4) + round256(P * 8) + round256(P / TILE * 32) + round256(P * 16) +
           2 * round256(P * 32) + round256(P * 4);
}

size_t ws_bytes(uint64_t S, uint64_t log_cap, SplitGrids grid) {
    const uint64_t P = padded(S);
    return common_bytes(P) + round256(log_cap * 12) + 256 + round256(part_bytes(P, grid));
}

NbWs carve(void* base, uint64_t S, uint64_t log_cap, SplitGrids grid) {
    const uint64_t P = padded(S);
    uint8_t* p = static_cast<uint8_t*>(base);
    NbWs w;
    carve_common(p, P, w);
    w.log = reinterpret_cast<int32_t*>(p);
    p += round256(log_cap * 12);
    w.log_n = reinterpret_cast<dsr_u64*>(p);
    w.step = reinterpret_cast<dsr_u64*>(p + 8);
    w.n_live = reinterpret_cast<uint32_t*>(p + 16);
    w.npairs = reinterpret_cast<uint32_t*>(p + 20);
    p += 256;
    w.part = reinterpret_cast<float4*>(p);
    w.part64 = reinterpret_cast<D4*>(p);
    w.log_cap = log_cap;
    return w;
}

// The spatial sort of one order (POST: the updated positions).
template <bool POST>
void launch_sort(dsr_heap* h, const NbArgs& a, cudaStream_t s) {
    const unsigned ctas = (unsigned)(h->sm_count * 4);
    k_cell_count<POST><<<ctas, 256, 0, s>>>(h->dev, a.ws);
    k_cell_sum<<<SCAN_CTAS, 1024, 0, s>>>(a.ws);
    k_cell_scan<<<SCAN_CTAS, 1024, 0, s>>>(a.ws, POST ? 1 : 0);
    k_cell_place<POST><<<ctas, 256, 0, s>>>(h->dev, a.ws);
    k_cell_order<POST><<<NKEYS / 256, 256, 0, s>>>(h->dev, a.ws);
}

// One step. `split`: the split force kernels with their grids (else the
// unsplit ones, for the allocation-free step); P: padded positions.
void launch_step(dsr_heap* h, const NbArgs& a, const SplitGrids* split, uint64_t P, cudaStream_t s) {
    const unsigned ctas = (unsigned)(h->sm_count * 4);
    const bool f64 = a.p.pair_precision == DSR_NBODY_PAIRS_FP64;
    const bool soft = a.p.eps * a.p.eps >= (double)FLT_MIN;
    dsr__launch_scan(h, BODY, s);
    launch_sort<false>(h, a, s);
    k_gather<<<ctas, TILE, 0, s>>>(h->dev, a.ws);
    uint32_t grid = 0;
    if (split) {
        grid = f64 ? split->force64 : split->force;
        if (f64)
            k_force_part64<<<grid, TILE, 0, s>>>(h->dev, a);
        else if (soft)
            k_force_part<true><<<grid, TILE, 0, s>>>(h->dev, a);
        else
            k_force_part<false><<<grid, TILE, 0, s>>>(h->dev, a);
    } else {
        const unsigned tiles = (unsigned)(P / TILE);
        if (f64)
            k_force64<<<tiles, TILE, 0, s>>>(h->dev, a);
        else
            k_force<<<tiles, TILE, 0, s>>>(h->dev, a);
    }
    k_update<<<ctas, UPDATE_THREADS, 0, s>>>(h->dev, a, grid);
    launch_sort<true>(h, a, s);
    k_partner<<<ctas, 256, 0, s>>>(h->dev, a);
    k_merge<<<ctas, 256, 0, s>>>(h->dev, a);
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
    if (heap->layout.n_blocks * 64 > 0x7FFFFFFFull) return DSR_E_INVALID;
    dsr_nbody* nb = new dsr_nbody;
    nb->heap = heap;
    nb->S = heap->layout.n_blocks * 64;
    nb->grid = split_grids(heap);
    nb->args.ws = carve(workspace_dev, nb->S, log_cap, nb->grid);
    nb->args.ws.K = cells_per_axis(*p);
    nb->args.p = *p;
    cudaStream_t s = dsr__stream(stream);
    cudaError_t e = cudaMemsetAsync(nb->args.ws.log_n, 0, 24, s);
    if (!e) e = cudaMemsetAsync(nb->args.ws.ccount, 0, NKEYS * 4, s);
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
    for (int i = 0; i < n_steps; ++i) {
        launch_step(nb->heap, nb->args, &nb->grid, padded(nb->S), s);
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
// Allocation-free step. The scratch of a step (the cell counts and offsets,
// the sorted state before and after the update, handles, partners and the
// far-field sums) lives in this file-scope device array instead of a
// caller-allocated workspace, for callers that cannot call cudaMalloc.
// Every GPU that loads the library holds the array until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr uint64_t kNoallocP = (DSR_NOALLOC_MAX_SLOTS + ROW - 1) / ROW * ROW;

struct NoallocScratch {
    uint32_t ccount[NKEYS];  // zero at load; every sort leaves it zero
    uint32_t coff[NKEYS + 1];
    uint32_t coff2[NKEYS + 1];
    uint32_t csum[SCAN_CTAS];
    uint32_t ckey[kNoallocP];
    uint32_t perm[kNoallocP];
    uint32_t perm2[kNoallocP];
    float4 pos[kNoallocP];
    D4 pd[kNoallocP];
    int32_t id[kNoallocP];
    dsr_u64 sref[kNoallocP];
    float4 tbox[kNoallocP / TILE * 2];
    float4 npos[kNoallocP];
    D4 npd[kNoallocP];
    D4 nvd[kNoallocP];
    int32_t partner[kNoallocP];
    D4 part[kNoallocP];  // far-field sums: FP32 (as float4) or FP64
    uint32_t n_live;
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
    a.ws.ccount = sc->ccount;
    a.ws.coff = sc->coff;
    a.ws.coff2 = sc->coff2;
    a.ws.csum = sc->csum;
    a.ws.ckey = sc->ckey;
    a.ws.perm = sc->perm;
    a.ws.perm2 = sc->perm2;
    a.ws.n_live = &sc->n_live;
    a.ws.npairs = &sc->npairs;
    a.ws.pos = sc->pos;
    a.ws.pd = sc->pd;
    a.ws.id = sc->id;
    a.ws.sref = sc->sref;
    a.ws.tbox = sc->tbox;
    a.ws.npos = sc->npos;
    a.ws.npd = sc->npd;
    a.ws.nvd = sc->nvd;
    a.ws.partner = sc->partner;
    a.ws.part = reinterpret_cast<float4*>(sc->part);  // one slice: the unsplit force kernels
    a.ws.part64 = sc->part;
    a.ws.log = static_cast<int32_t*>(log_dev);
    a.ws.log_n = static_cast<dsr_u64*>(log_count_dev);
    a.ws.step = &sc->step;
    a.ws.log_cap = log_cap;
    a.ws.K = cells_per_axis(*p);
    cudaStream_t s = dsr__stream(stream);
    // The array keeps the previous call's contents. The step counter is the
    // only value a step reads before writing it; the cell counts are zero
    // when the library is loaded and every sort returns them to zero.
    k_set_u64<<<1, 1, 0, s>>>(&sc->step, step0);
    for (int i = 0; i < n_steps; ++i) launch_step(heap, a, nullptr, padded(S), s);
    return dsr__check_launch("dsr_nbody_step_noalloc");
}
