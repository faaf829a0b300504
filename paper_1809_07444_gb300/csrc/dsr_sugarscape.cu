// Sugarscape as an SMMO program (Fig. 6f; Epstein and Axtell's movement rule
// M, growback rule G_alpha and replacement rule R): Agent objects on a
// W x H torus of sugar cells, four do-alls per step.
//
//   A1 choose:  the candidate cell with the most sugar among the agent's own
//               cell and the free cells up to `vision` away in the order N,
//               E, S, W; then the nearest; then (r >> 32) mod k with
//               r = rand(seed, 12, t, own cell). Another cell is claimed
//               (atomicMin of the own cell index).
//   A2 move:    the winner of a claim moves (and resets the claim); every
//               agent harvests its cell, pays its metabolism, ages, and is
//               marked dead when its sugar is below 0 or its age reached
//               max_age.
//   A3 claim:   a dead agent draws c = (rand(seed, 13, t, own) >> 32) mod
//               (W * H) and claims c if no agent occupies it.
//   A4 replace: a dead agent creates a new agent (age 0, attributes drawn
//               from streams 8..11 keyed on the new cell) at c if it won c,
//               else in its own cell, and deletes itself.
// Sugar grows back lazily: a cell keeps the step of its last harvest h, and
// its sugar at the start of step t is min(cap, alpha * (t - h)) (cap if
// never harvested), which equals applying G_alpha at the end of every step,
// without a pass over all cells. A cell is one 32-bit word: bit 31 set
// while an agent (alive or dead) is on it, bits 28-30 its capacity, bits
// 0-27 its last harvest step + 1 (0: never), so that the choice reads one
// word per cell in sight. Steps are limited to 2^28 - 2.
#include <climits>

#include "dsr_apps.h"
#include "dsr_internal.cuh"

namespace {
enum { AGENT = 0 };
enum { F_X, F_Y, F_SUGAR, F_METAB, F_VISION, F_AGE, F_MAXAGE, F_DEAD, NF };
enum { EV_MOVES, EV_STARVED, EV_AGED, EV_AWAY, EV_HARVEST, N_EV };
constexpr uint32_t NO_CLAIM = 0xFFFFFFFFu;
constexpr uint32_t OCC = 0x80000000u, CAP_SHIFT = 28, STEP_MASK = 0x0FFFFFFFu;

struct SugarWs {
    uint32_t* cell;      // [n] occupancy bit, capacity, last harvest step + 1
    uint32_t* claim;     // [n] A1 claims (lowest own cell wins), NO_CLAIM
    uint32_t* claim2;    // [n] A3 claims
    uint32_t* intent;    // [heap slots] A1 target of each agent slot
    dsr_u64 n_slots;
    dsr_u64* events;     // [DSR_CTR_SLOTS][N_EV] cumulative, one row per SM slot
};

struct SugarArgs {
    SugarWs ws;
    dsr_sugarscape_params p;
    int64_t step;
};

__device__ __forceinline__ int32_t* fld(const dsr_dev_heap& H, dsr_ref r, int f) {
    return dsr_field<int32_t>(H, AGENT, r, f);
}

__device__ __forceinline__ int32_t sugar_of(const SugarArgs& a, uint32_t st) {
    const int32_t cap = (int32_t)((st >> CAP_SHIFT) & 7u);
    const uint32_t h1 = st & STEP_MASK;
    if (h1 == 0) return cap;  // never harvested
    const int64_t d = a.step - (int64_t)(h1 - 1);  // steps of growback since the harvest
    if (d >= cap) return cap;        // alpha >= 1: full again
    const int64_t v = (int64_t)a.p.alpha * d;
    return v < cap ? (int32_t)v : cap;
}

__device__ __forceinline__ int32_t draw(const SugarArgs& a, dsr_u64 stream, int64_t c, int32_t lo, int32_t hi) {
    const dsr_u64 r = dsr_rand(a.p.seed, stream, (dsr_u64)a.step, (dsr_u64)c) >> 32;
    return lo + (int32_t)(r % (dsr_u64)(hi - lo + 1));
}

// Sum of a per-lane count over the calling lanes, one atomic per warp, on
// the row of the warp's SM (rows spread the atomics over many addresses).
__device__ __forceinline__ void count_event(const SugarArgs& a, int k, unsigned v) {
    const unsigned act = __activemask();
    v = __reduce_add_sync(act, v);
    if (v && dsr_lane() == (unsigned)(__ffs(act) - 1)) {
        unsigned smid;
        asm("mov.u32 %0, %%smid;" : "=r"(smid));
        atomicAdd(a.ws.events + (smid % DSR_CTR_SLOTS) * N_EV + k, (dsr_u64)v);
    }
}

struct MChoose {
    typedef SugarArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        const int32_t x = *fld(H, self, F_X), y = *fld(H, self, F_Y), vision = *fld(H, self, F_VISION);
        const int32_t W = a.p.W, Hh = a.p.H;
        const int64_t own = (int64_t)y * W + x;
        int32_t best = sugar_of(a, a.ws.cell[own]), best_d = 0;
        unsigned dirs = 0;  // directions (bit 0 N, 1 E, 2 S, 3 W) of the candidates at distance best_d
        for (int32_t d = 1; d <= vision; ++d) {
            const int32_t yn = y - d < 0 ? y - d + Hh : y - d, ys = y + d >= Hh ? y + d - Hh : y + d;
            const int32_t xe = x + d >= W ? x + d - W : x + d, xw = x - d < 0 ? x - d + W : x - d;
            const uint32_t st[4] = {a.ws.cell[(int64_t)yn * W + x], a.ws.cell[(int64_t)y * W + xe],
                                    a.ws.cell[(int64_t)ys * W + x], a.ws.cell[(int64_t)y * W + xw]};
#pragma unroll
            for (int dir = 0; dir < 4; ++dir) {
                if (st[dir] & OCC) continue;
                const int32_t v = sugar_of(a, st[dir]);
                if (v > best) {
                    best = v;
                    best_d = d;
                    dirs = 1u << dir;
                } else if (v == best && d == best_d) {
                    dirs |= 1u << dir;
                }
            }
        }
        int64_t t = own;
        if (best_d > 0) {
            const int k = __popc(dirs);
            int pick = 0;
            if (k > 1) pick = (int)((dsr_rand(a.p.seed, 12, (dsr_u64)a.step, (dsr_u64)own) >> 32) % (dsr_u64)k);
            const int dir = dsr_nth_bit(dirs, pick);
            const int32_t d = best_d;
            if (dir == 0) t = (int64_t)(y - d < 0 ? y - d + Hh : y - d) * W + x;
            if (dir == 1) t = (int64_t)y * W + (x + d >= W ? x + d - W : x + d);
            if (dir == 2) t = (int64_t)(y + d >= Hh ? y + d - Hh : y + d) * W + x;
            if (dir == 3) t = (int64_t)y * W + (x - d < 0 ? x - d + W : x - d);
        }
        if (dsr_check(self < a.ws.n_slots, H.err, H.dbg, 8, self)) a.ws.intent[self] = (uint32_t)t;
        if (t != own) atomicMin(a.ws.claim + t, (uint32_t)own);
    }
};

struct MMove {
    typedef SugarArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        if (!dsr_check(self < a.ws.n_slots, H.err, H.dbg, 8, self)) return;
        const int32_t x = *fld(H, self, F_X), y = *fld(H, self, F_Y);
        const int64_t own = (int64_t)y * a.p.W + x;
        const int64_t t = a.ws.intent[self];
        int64_t c = own;
        unsigned moved = 0;
        if (t != own && a.ws.claim[t] == (uint32_t)own) {
            a.ws.claim[t] = NO_CLAIM;  // only the winner matches, so the reset cannot make a loser win
            a.ws.cell[own] &= ~OCC;     // this agent is the only writer of both cells in this do-all
            a.ws.cell[t] |= OCC;
            *fld(H, self, F_X) = (int32_t)(t % a.p.W);
            *fld(H, self, F_Y) = (int32_t)(t / a.p.W);
            c = t;
            moved = 1;
        }
        const uint32_t st = a.ws.cell[c];
        const int32_t got = sugar_of(a, st);
        a.ws.cell[c] = (st & ~STEP_MASK) | (uint32_t)(a.step + 1);
        const int32_t sugar = *fld(H, self, F_SUGAR) + got - *fld(H, self, F_METAB);
        const int32_t age = *fld(H, self, F_AGE) + 1;
        *fld(H, self, F_SUGAR) = sugar;
        *fld(H, self, F_AGE) = age;
        const unsigned starved = sugar < 0, aged = !starved && age >= *fld(H, self, F_MAXAGE);
        if (starved || aged) *fld(H, self, F_DEAD) = 1;
        count_event(a, EV_MOVES, moved);
        count_event(a, EV_STARVED, starved);
        count_event(a, EV_AGED, aged);
        count_event(a, EV_HARVEST, (unsigned)got);
    }
};

__device__ __forceinline__ int64_t replacement_cell(const SugarArgs& a, int64_t own) {
    const dsr_u64 n = (dsr_u64)a.p.W * a.p.H;
    return (int64_t)((dsr_rand(a.p.seed, 13, (dsr_u64)a.step, (dsr_u64)own) >> 32) % n);
}

struct MReplaceClaim {
    typedef SugarArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        if (!*fld(H, self, F_DEAD)) return;
        const int64_t own = (int64_t)*fld(H, self, F_Y) * a.p.W + *fld(H, self, F_X);
        const int64_t c = replacement_cell(a, own);
        if (!(a.ws.cell[c] & OCC)) atomicMin(a.ws.claim2 + c, (uint32_t)own);
    }
};

struct MReplace {
    typedef SugarArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        if (!*fld(H, self, F_DEAD)) return;
        const int64_t own = (int64_t)*fld(H, self, F_Y) * a.p.W + *fld(H, self, F_X);
        const int64_t c = replacement_cell(a, own);
        int64_t at = own;
        unsigned away = 0;
        if (a.ws.claim2[c] == (uint32_t)own) {
            a.ws.claim2[c] = NO_CLAIM;
            a.ws.cell[own] &= ~OCC;
            a.ws.cell[c] |= OCC;
            at = c;
            away = 1;
        }
        count_event(a, EV_AWAY, away);
        dsr_delete(H, self);  // first, so that the new agent may take the slot
        const dsr_ref r = dsr_new(H, AGENT, self);  // tried first: the block just given a free slot
        if (r == DSR_NULL) return;  // out of memory: DSR_ERR_OOM is set
        *fld(H, r, F_X) = (int32_t)(at % a.p.W);
        *fld(H, r, F_Y) = (int32_t)(at / a.p.W);
        *fld(H, r, F_SUGAR) = draw(a, 8, at, a.p.endow_lo, a.p.endow_hi);
        *fld(H, r, F_METAB) = draw(a, 9, at, a.p.metab_lo, a.p.metab_hi);
        *fld(H, r, F_VISION) = draw(a, 10, at, a.p.vision_lo, a.p.vision_hi);
        *fld(H, r, F_AGE) = 0;
        *fld(H, r, F_MAXAGE) = draw(a, 11, at, a.p.age_lo, a.p.age_hi);
        *fld(H, r, F_DEAD) = 0;
    }
};

// One thread per initial agent (agents0[i] = x, y, sugar, metabolism,
// vision, age, max_age; distinct cells).
__global__ void k_sugar_init(const __grid_constant__ dsr_dev_heap H, const int32_t* agents0, int64_t n_agents,
                             SugarWs ws, int32_t W) {
    const int64_t n32 = (n_agents + 31) & ~31ll;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n32; i += (int64_t)gridDim.x * blockDim.x) {
        __syncwarp();
        if (i >= n_agents) continue;
        const int32_t* src = agents0 + 7 * i;
        const dsr_ref r = dsr_new(H, AGENT);
        if (r == DSR_NULL) continue;
        for (int f = 0; f < 7; ++f) *fld(H, r, f) = src[f];
        *fld(H, r, F_DEAD) = 0;
        ws.cell[(int64_t)src[1] * W + src[0]] |= OCC;
    }
}

// Cells from the capacities: unoccupied, never harvested.
__global__ void k_sugar_fill(uint32_t* cell, const uint8_t* cap, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        cell[i] = (uint32_t)(cap[i] & 7u) << CAP_SHIFT;
}

__global__ void k_sugar_read(SugarArgs a, int32_t* out) {
    const int64_t n = (int64_t)a.p.W * a.p.H;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = sugar_of(a, a.ws.cell[i]);
}

const int kAgentFields[NF] = {4, 4, 4, 4, 4, 4, 4, 4};

bool heap_matches(const dsr_heap* h) {
    const dsr_layout& L = h->layout;
    if (L.n_types < 1 || L.n_fields[AGENT] != NF) return false;
    for (int f = 0; f < NF; ++f)
        if (L.field_bytes[AGENT][f] != 4) return false;
    return true;
}

bool params_ok(const dsr_sugarscape_params* p) {
    return p && p->alpha >= 1 && p->vision_lo >= 1 && p->vision_hi >= p->vision_lo && p->vision_hi <= 64 &&
           p->W >= 2 * p->vision_hi + 1 && p->H >= 2 * p->vision_hi + 1 && (int64_t)p->W * p->H < (1ll << 31) &&
           p->metab_hi >= p->metab_lo && p->endow_hi >= p->endow_lo && p->age_lo >= 1 && p->age_hi >= p->age_lo;
}

size_t r256(size_t x) { return (x + 255) / 256 * 256; }

size_t ws_bytes(const dsr_sugarscape_params& p, dsr_u64 slots) {
    const size_t n = (size_t)p.W * p.H;
    return 3 * r256(n * 4) + r256(slots * 4) + r256(DSR_CTR_SLOTS * N_EV * 8);
}

SugarWs carve(void* base, const dsr_sugarscape_params& p, dsr_u64 slots) {
    const size_t n = (size_t)p.W * p.H;
    uint8_t* q = static_cast<uint8_t*>(base);
    SugarWs w;
    w.cell = reinterpret_cast<uint32_t*>(q);
    q += r256(n * 4);
    w.claim = reinterpret_cast<uint32_t*>(q);
    q += r256(n * 4);
    w.claim2 = reinterpret_cast<uint32_t*>(q);
    q += r256(n * 4);
    w.intent = reinterpret_cast<uint32_t*>(q);
    q += r256(slots * 4);
    w.events = reinterpret_cast<dsr_u64*>(q);
    w.n_slots = slots;
    return w;
}
}  // namespace

struct dsr_sugarscape {
    dsr_heap* heap;
    SugarArgs args;
};

extern "C" int dsr_sugarscape_types(dsr_type_desc* out) {
    if (!out) return DSR_E_INVALID;
    out[0] = dsr_type_desc{"Agent", NF, kAgentFields};
    return DSR_OK;
}

extern "C" int dsr_sugarscape_workspace_bytes(const dsr_heap* heap, const dsr_sugarscape_params* p, size_t* out) {
    if (!heap || !out || !params_ok(p)) return DSR_E_INVALID;
    *out = ws_bytes(*p, heap->layout.n_blocks * 64);
    return DSR_OK;
}

extern "C" int dsr_sugarscape_create(dsr_heap* heap, const dsr_sugarscape_params* p, const void* cap_dev,
                                     const void* agents0_dev, int64_t n_agents, void* workspace_dev, void* stream,
                                     dsr_sugarscape** out) {
    if (!heap || !cap_dev || (n_agents && !agents0_dev) || n_agents < 0 || !workspace_dev || !out || !params_ok(p) ||
        !heap_matches(heap))
        return DSR_E_INVALID;
    if (reinterpret_cast<uintptr_t>(workspace_dev) & 255) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    const dsr_u64 slots = heap->layout.n_blocks * 64;
    const int64_t n = (int64_t)p->W * p->H;
    dsr_sugarscape* g = new dsr_sugarscape;
    g->heap = heap;
    g->args.ws = carve(workspace_dev, *p, slots);
    g->args.p = *p;
    g->args.step = 0;
    SugarWs& w = g->args.ws;
    cudaError_t e = cudaMemsetAsync(w.claim, 0xFF, (size_t)n * 4, s);
    if (!e) e = cudaMemsetAsync(w.claim2, 0xFF, (size_t)n * 4, s);
    if (!e) e = cudaMemsetAsync(w.events, 0, DSR_CTR_SLOTS * N_EV * 8, s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_sugarscape_create");
        delete g;
        return DSR_E_CUDA;
    }
    const int ctas = heap->sm_count * 4;
    k_sugar_fill<<<ctas, 256, 0, s>>>(w.cell, static_cast<const uint8_t*>(cap_dev), n);
    if (n_agents) {
        int64_t c2 = (n_agents + 255) / 256;
        if (c2 > heap->sm_count * 8) c2 = heap->sm_count * 8;
        k_sugar_init<<<(unsigned)c2, 256, 0, s>>>(heap->dev, static_cast<const int32_t*>(agents0_dev), n_agents, w,
                                                    p->W);
    }
    const int rc = dsr__check_launch("k_sugar_init");
    if (rc) {
        delete g;
        return rc;
    }
    *out = g;
    return DSR_OK;
}

extern "C" int dsr_sugarscape_step(dsr_sugarscape* g, int n_steps, void* stream) {
    if (!g || n_steps < 0 || g->args.step + n_steps > (int64_t)STEP_MASK - 1) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    for (int i = 0; i < n_steps; ++i) {
        // A1-A4 visit the same live set (nothing is created or deleted before
        // A4), so A2-A4 reuse A1's block list.
        int rc = dsr__doall<MChoose>(g->heap, AGENT, g->args, s, true, nullptr, nullptr, 3);
        if (!rc) rc = dsr__doall<MMove>(g->heap, AGENT, g->args, s, false, nullptr, nullptr, 2);
        if (!rc) rc = dsr__doall<MReplaceClaim>(g->heap, AGENT, g->args, s, false, nullptr, nullptr, 1);
        if (!rc) rc = dsr__doall<MReplace>(g->heap, AGENT, g->args, s, false);
        if (rc) return rc;
        g->args.step += 1;
    }
    return DSR_OK;
}

extern "C" int dsr_sugarscape_events(dsr_sugarscape* g, void* stream, uint64_t* out) {
    if (!g || !out) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    static thread_local dsr_u64 rows[DSR_CTR_SLOTS * N_EV];
    cudaError_t e = cudaMemcpyAsync(rows, g->args.ws.events, sizeof rows, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_sugarscape_events");
        return DSR_E_CUDA;
    }
    for (int k = 0; k < N_EV; ++k) {
        out[k] = 0;
        for (int r = 0; r < DSR_CTR_SLOTS; ++r) out[k] += rows[r * N_EV + k];
    }
    return DSR_OK;
}

extern "C" int dsr_sugarscape_sugar(dsr_sugarscape* g, void* out_dev, void* stream) {
    if (!g || !out_dev) return DSR_E_INVALID;
    k_sugar_read<<<g->heap->sm_count * 4, 256, 0, dsr__stream(stream)>>>(g->args, static_cast<int32_t*>(out_dev));
    return dsr__check_launch("k_sugar_read");
}

extern "C" int dsr_sugarscape_destroy(dsr_sugarscape* g) {
    delete g;
    return DSR_OK;
}
