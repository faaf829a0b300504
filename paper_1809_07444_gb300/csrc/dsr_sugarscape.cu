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
// without a pass over all cells.
#include <climits>

#include "dsr_apps.h"
#include "dsr_internal.cuh"

namespace {
enum { AGENT = 0 };
enum { F_X, F_Y, F_SUGAR, F_METAB, F_VISION, F_AGE, F_MAXAGE, F_DEAD, NF };
enum { EV_MOVES, EV_STARVED, EV_AGED, EV_AWAY, EV_HARVEST, N_EV };
constexpr int32_t NEVER = INT_MIN;       // harvest step of a cell never harvested
constexpr uint32_t NO_CLAIM = 0xFFFFFFFFu;

struct SugarWs {
    const uint8_t* cap;  // [n] capacity
    uint8_t* occ;        // [n] 1 = an agent (alive or dead) is on the cell
    int32_t* harvested;  // [n] step of the last harvest, NEVER if none
    uint32_t* claim;     // [n] A1 claims (lowest own cell wins), NO_CLAIM
    uint32_t* claim2;    // [n] A3 claims
    uint32_t* intent;    // [heap slots] A1 target of each agent slot
    dsr_u64 n_slots;
    dsr_u64* events;     // [N_EV] cumulative
};

struct SugarArgs {
    SugarWs ws;
    dsr_sugarscape_params p;
    int64_t step;
};

__device__ __forceinline__ int32_t* fld(const dsr_dev_heap& H, dsr_ref r, int f) {
    return dsr_field<int32_t>(H, AGENT, r, f);
}

__device__ __forceinline__ int32_t sugar_at(const SugarArgs& a, int64_t c) {
    const int32_t cap = a.ws.cap[c];
    const int32_t h = a.ws.harvested[c];
    if (h == NEVER) return cap;
    const int64_t d = a.step - h;  // steps of growback since the harvest
    if (d >= cap) return cap;        // alpha >= 1: full again
    const int64_t v = (int64_t)a.p.alpha * d;
    return v < cap ? (int32_t)v : cap;
}

__device__ __forceinline__ int32_t draw(const SugarArgs& a, dsr_u64 stream, int64_t c, int32_t lo, int32_t hi) {
    const dsr_u64 r = dsr_rand(a.p.seed, stream, (dsr_u64)a.step, (dsr_u64)c) >> 32;
    return lo + (int32_t)(r % (dsr_u64)(hi - lo + 1));
}

// Sum of a per-lane count over the calling lanes, one atomic per warp.
__device__ __forceinline__ void count_event(const SugarArgs& a, int k, unsigned v) {
    const unsigned act = __activemask();
    v = __reduce_add_sync(act, v);
    if (v && dsr_lane() == (unsigned)(__ffs(act) - 1)) atomicAdd(a.ws.events + k, (dsr_u64)v);
}

struct MChoose {
    typedef SugarArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        const int32_t x = *fld(H, self, F_X), y = *fld(H, self, F_Y), vision = *fld(H, self, F_VISION);
        const int32_t W = a.p.W, Hh = a.p.H;
        const int64_t own = (int64_t)y * W + x;
        int32_t best = sugar_at(a, own), best_d = 0, k = 1;
        int64_t cand[4] = {own, own, own, own};
        for (int32_t d = 1; d <= vision; ++d) {
#pragma unroll
            for (int dir = 0; dir < 4; ++dir) {  // N, E, S, W
                int32_t cx = x, cy = y;
                if (dir == 0) cy = y - d < 0 ? y - d + Hh : y - d;
                if (dir == 1) cx = x + d >= W ? x + d - W : x + d;
                if (dir == 2) cy = y + d >= Hh ? y + d - Hh : y + d;
                if (dir == 3) cx = x - d < 0 ? x - d + W : x - d;
                const int64_t c = (int64_t)cy * W + cx;
                if (a.ws.occ[c]) continue;
                const int32_t v = sugar_at(a, c);
                if (v > best) {
                    best = v;
                    best_d = d;
                    k = 1;
                    cand[0] = c;
                } else if (v == best && d == best_d) {
                    cand[k++] = c;
                }
            }
        }
        int64_t t = cand[0];
        if (k > 1) {
            const dsr_u64 r = dsr_rand(a.p.seed, 12, (dsr_u64)a.step, (dsr_u64)own) >> 32;
            const int32_t pick = (int32_t)(r % (dsr_u64)k);
            t = pick == 1 ? cand[1] : pick == 2 ? cand[2] : pick == 3 ? cand[3] : cand[0];
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
            a.ws.occ[own] = 0;
            a.ws.occ[t] = 1;
            *fld(H, self, F_X) = (int32_t)(t % a.p.W);
            *fld(H, self, F_Y) = (int32_t)(t / a.p.W);
            c = t;
            moved = 1;
        }
        const int32_t got = sugar_at(a, c);
        a.ws.harvested[c] = (int32_t)a.step;
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
        if (!a.ws.occ[c]) atomicMin(a.ws.claim2 + c, (uint32_t)own);
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
            a.ws.occ[own] = 0;
            a.ws.occ[c] = 1;
            at = c;
            away = 1;
        }
        count_event(a, EV_AWAY, away);
        const dsr_ref r = dsr_new(H, AGENT);
        dsr_delete(H, self);
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
        ws.occ[(int64_t)src[1] * W + src[0]] = 1;
    }
}

__global__ void k_sugar_fill(int32_t* harvested, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        harvested[i] = NEVER;
}

__global__ void k_sugar_read(SugarArgs a, int32_t* out) {
    const int64_t n = (int64_t)a.p.W * a.p.H;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = sugar_at(a, i);
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
    return 2 * r256(n) + 3 * r256(n * 4) + r256(slots * 4) + 256;
}

SugarWs carve(void* base, const dsr_sugarscape_params& p, dsr_u64 slots) {
    const size_t n = (size_t)p.W * p.H;
    uint8_t* q = static_cast<uint8_t*>(base);
    SugarWs w;
    w.cap = q;
    q += r256(n);
    w.occ = q;
    q += r256(n);
    w.harvested = reinterpret_cast<int32_t*>(q);
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
    cudaError_t e = cudaMemcpyAsync(const_cast<uint8_t*>(w.cap), cap_dev, (size_t)n, cudaMemcpyDeviceToDevice, s);
    if (!e) e = cudaMemsetAsync(w.occ, 0, (size_t)n, s);
    if (!e) e = cudaMemsetAsync(w.claim, 0xFF, (size_t)n * 4, s);
    if (!e) e = cudaMemsetAsync(w.claim2, 0xFF, (size_t)n * 4, s);
    if (!e) e = cudaMemsetAsync(w.events, 0, 256, s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_sugarscape_create");
        delete g;
        return DSR_E_CUDA;
    }
    const int ctas = heap->sm_count * 4;
    k_sugar_fill<<<ctas, 256, 0, s>>>(w.harvested, n);
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
    if (!g || n_steps < 0) return DSR_E_INVALID;
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
    cudaError_t e = cudaMemcpyAsync(out, g->args.ws.events, N_EV * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_sugarscape_events");
        return DSR_E_CUDA;
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
