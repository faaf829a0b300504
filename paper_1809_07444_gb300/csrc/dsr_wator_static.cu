// Wa-tor without dynamic allocation: the "Baseline AOS/SOA" comparators of
// Section 4 (variants of an application with no dynamic allocation). The
// agents live in per-cell arrays, every phase is a kernel over all cells, and
// a move copies an agent's data from its cell to the target cell. The rules,
// the random draws and the claim keys are those of dsr_wator.cu, so a run
// gives the same state, step by step, as the allocator-based form (and the
// oracle). Two layouts: SOA (one array per field) and AOS (one struct per
// cell).
#include "dsr_apps.h"
#include "dsr_internal.cuh"

namespace {
enum : uint8_t { EMPTY = 0, FISH = 1, SHARK = 2 };
constexpr uint32_t NONE = 0xFFFFFFFFu;  // no agent of the phase's kind here
constexpr uint32_t STAY = 0xFFFFFFFEu;  // an agent with no candidate cell

struct AosCell {
    int32_t timer;
    int32_t energy;
    uint8_t kind;
    uint8_t pad[3];
};

// Field access for the two layouts.
struct Soa {
    uint8_t* kind_;
    int32_t* timer_;
    int32_t* energy_;
    __device__ uint8_t kind(uint32_t c) const { return kind_[c]; }
    __device__ int32_t& timer(uint32_t c) const { return timer_[c]; }
    __device__ int32_t& energy(uint32_t c) const { return energy_[c]; }
    __device__ void set_kind(uint32_t c, uint8_t k) const { kind_[c] = k; }
};
struct Aos {
    AosCell* cell;
    __device__ uint8_t kind(uint32_t c) const { return cell[c].kind; }
    __device__ int32_t& timer(uint32_t c) const { return cell[c].timer; }
    __device__ int32_t& energy(uint32_t c) const { return cell[c].energy; }
    __device__ void set_kind(uint32_t c, uint8_t k) const { cell[c].kind = k; }
};

struct StaticWs {
    dsr_u64* claim;      // lowest claim key of the current phase (never reset)
    uint32_t* intent;    // target, STAY or NONE
    dsr_u64* visits;     // agents visited by the phase kernels
    dsr_wator_params p;
};

__device__ __forceinline__ dsr_u64 claim_key(dsr_u64 t, unsigned ph, uint32_t c) {
    return ((0xFFFFFFFFull - (2 * t + ph)) << 32) | c;
}

__device__ __forceinline__ void neighbours(uint32_t c, int W, int H, uint32_t nb[4]) {
    const int x = (int)(c % (uint32_t)W), y = (int)(c / (uint32_t)W);
    nb[0] = (uint32_t)((y == 0 ? H - 1 : y - 1) * W + x);  // N
    nb[1] = (uint32_t)(y * W + (x == W - 1 ? 0 : x + 1));  // E
    nb[2] = (uint32_t)((y == H - 1 ? 0 : y + 1) * W + x);  // S
    nb[3] = (uint32_t)(y * W + (x == 0 ? W - 1 : x - 1));  // W
}

__device__ __forceinline__ int pick(unsigned m, unsigned k) {
    for (int d = 0; d < 4; ++d)
        if ((m >> d) & 1u) {
            if (k == 0) return d;
            --k;
        }
    return 0;
}

// One visit per calling lane, one atomic per warp.
__device__ __forceinline__ void count_visit(dsr_u64* visits) {
    const unsigned act = __activemask();
    if ((threadIdx.x & 31) == (unsigned)(__ffs(act) - 1)) atomicAdd(visits, (dsr_u64)__popc(act));
}

#define CELL_LOOP(n)                                                                               \
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < (n); c += gridDim.x * blockDim.x)

template <class L>
__global__ void k_st_init(L A, StaticWs S, const uint8_t* kind0) {
    const uint32_t n = (uint32_t)S.p.W * (uint32_t)S.p.H;
    CELL_LOOP(n) {
        const uint8_t k = kind0[c] == 1 ? FISH : kind0[c] == 2 ? SHARK : EMPTY;
        A.set_kind(c, k);
        A.timer(c) = 0;
        A.energy(c) = k == SHARK ? S.p.shark_energy0 : 0;
        S.claim[c] = ~0ull;
        S.intent[c] = NONE;
    }
}

// F1: fish age, pick an empty neighbour, claim it.
template <class L>
__global__ void k_st_f1(L A, StaticWs S, dsr_u64 t) {
    const uint32_t n = (uint32_t)S.p.W * (uint32_t)S.p.H;
    CELL_LOOP(n) {
        if (A.kind(c) != FISH) continue;
        count_visit(S.visits);
        A.timer(c) += 1;
        uint32_t nb[4];
        neighbours(c, S.p.W, S.p.H, nb);
        unsigned m = 0;
#pragma unroll
        for (int d = 0; d < 4; ++d) m |= (A.kind(nb[d]) == EMPTY ? 1u : 0u) << d;
        uint32_t tgt = STAY;
        if (m) {
            tgt = nb[pick(m, (unsigned)(dsr_rand(S.p.seed, 0, t, c) % (dsr_u64)__popc(m)))];
            atomicMin(S.claim + tgt, claim_key(t, 0, c));
        }
        S.intent[c] = tgt;
    }
}

// F2: winners move (the agent's data goes to the target cell) and breed.
// Only cells whose fish took part in F1 have an intent, so a fish that moved
// into a cell in this kernel is not processed again.
template <class L>
__global__ void k_st_f2(L A, StaticWs S, dsr_u64 t) {
    const uint32_t n = (uint32_t)S.p.W * (uint32_t)S.p.H;
    CELL_LOOP(n) {
        const uint32_t tgt = S.intent[c];
        if (tgt == NONE) continue;
        count_visit(S.visits);
        S.intent[c] = NONE;
        if (tgt == STAY || S.claim[tgt] != claim_key(t, 0, c)) continue;
        const int32_t age = A.timer(c);
        A.set_kind(tgt, FISH);
        if (age >= S.p.fish_breed) {
            A.timer(tgt) = 0;
            A.timer(c) = 0;  // the newborn stays behind
        } else {
            A.timer(tgt) = age;
            A.set_kind(c, EMPTY);
        }
    }
}

// S0: starvation.
template <class L>
__global__ void k_st_s0(L A, StaticWs S) {
    const uint32_t n = (uint32_t)S.p.W * (uint32_t)S.p.H;
    CELL_LOOP(n) {
        if (A.kind(c) != SHARK) continue;
        count_visit(S.visits);
        if (--A.energy(c) <= 0) A.set_kind(c, EMPTY);
    }
}

// S1: sharks age, prefer a neighbouring fish, else an empty cell; claim it.
template <class L>
__global__ void k_st_s1(L A, StaticWs S, dsr_u64 t) {
    const uint32_t n = (uint32_t)S.p.W * (uint32_t)S.p.H;
    CELL_LOOP(n) {
        if (A.kind(c) != SHARK) continue;
        count_visit(S.visits);
        A.timer(c) += 1;
        uint32_t nb[4];
        neighbours(c, S.p.W, S.p.H, nb);
        unsigned mf = 0, me = 0;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const uint8_t k = A.kind(nb[d]);
            mf |= (k == FISH ? 1u : 0u) << d;
            me |= (k == EMPTY ? 1u : 0u) << d;
        }
        const unsigned m = mf ? mf : me;
        uint32_t tgt = STAY;
        if (m) {
            tgt = nb[pick(m, (unsigned)(dsr_rand(S.p.seed, 1, t, c) % (dsr_u64)__popc(m)))];
            atomicMin(S.claim + tgt, claim_key(t, 1, c));
        }
        S.intent[c] = tgt;
    }
}

// S2: winners move, eat and breed.
template <class L>
__global__ void k_st_s2(L A, StaticWs S, dsr_u64 t) {
    const uint32_t n = (uint32_t)S.p.W * (uint32_t)S.p.H;
    CELL_LOOP(n) {
        const uint32_t tgt = S.intent[c];
        if (tgt == NONE) continue;
        count_visit(S.visits);
        S.intent[c] = NONE;
        if (tgt == STAY || S.claim[tgt] != claim_key(t, 1, c)) continue;
        const int32_t age = A.timer(c);
        int32_t e = A.energy(c);
        if (A.kind(tgt) == FISH) e += S.p.shark_gain;
        A.set_kind(tgt, SHARK);
        A.energy(tgt) = e;
        if (age >= S.p.shark_breed) {
            A.timer(tgt) = 0;
            A.timer(c) = 0;  // the newborn stays behind
            A.energy(c) = S.p.shark_energy0;
        } else {
            A.timer(tgt) = age;
            A.set_kind(c, EMPTY);
        }
    }
}

// The object-state hash of dsr_heap_hash over the agents, as Fish {x, y,
// timer} and Shark {x, y, timer, energy}: out[0] fish, out[1] sharks.
template <class L>
__global__ void k_st_hash(L A, StaticWs S, dsr_u64* out) {
    const uint32_t n = (uint32_t)S.p.W * (uint32_t)S.p.H;
    CELL_LOOP(n) {
        const uint8_t k = A.kind(c);
        if (k == EMPTY) continue;
        const int T = k == FISH ? 0 : 1;
        const uint32_t w[4] = {c % (uint32_t)S.p.W, c / (uint32_t)S.p.W, (uint32_t)A.timer(c), (uint32_t)A.energy(c)};
        dsr_u64 h = dsr_mix64((dsr_u64)T + DSR_GAMMA);
        for (int f = 0; f < (T == 0 ? 3 : 4); ++f) h = dsr_mix64((h ^ (dsr_u64)w[f]) + DSR_GAMMA);
        atomicAdd(out + T, h);
    }
}

// Agents as SOA arrays: kind (0/1/2), timer, energy (0 for fish).
template <class L>
__global__ void k_st_state(L A, StaticWs S, uint8_t* kind, int32_t* timer, int32_t* energy) {
    const uint32_t n = (uint32_t)S.p.W * (uint32_t)S.p.H;
    CELL_LOOP(n) {
        const uint8_t k = A.kind(c);
        kind[c] = k;
        timer[c] = k == EMPTY ? 0 : A.timer(c);
        energy[c] = k == SHARK ? A.energy(c) : 0;
    }
}

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

bool params_ok(const dsr_wator_params* p) {
    return p && p->W >= 3 && p->H >= 3 && (int64_t)p->W * p->H < (1ll << 31) && p->fish_breed >= 0 &&
           p->shark_breed >= 0 && p->shark_energy0 >= 1;
}
}  // namespace

struct dsr_wator_static {
    int aos;
    Soa soa;
    Aos a;
    StaticWs ws;
    dsr_u64 t;
    int sm_count;
};

static size_t layout(int W, int H, int aos, size_t off[6]) {
    const size_t n = (size_t)W * H;
    size_t o = 0;
    if (aos) {
        off[0] = o;
        o += up256(n * sizeof(AosCell));
        off[1] = off[2] = 0;
    } else {
        off[0] = o;
        o += up256(n);
        off[1] = o;
        o += up256(n * 4);
        off[2] = o;
        o += up256(n * 4);
    }
    off[3] = o;  // claim
    o += up256(n * 8);
    off[4] = o;  // intent
    o += up256(n * 4);
    off[5] = o;  // visits
    o += 256;
    return o;
}

template <class L>
static int launch_step(dsr_wator_static* w, L A, cudaStream_t s) {
    const uint32_t n = (uint32_t)w->ws.p.W * (uint32_t)w->ws.p.H;
    unsigned ctas = (n + 255) / 256;
    if (ctas > (unsigned)w->sm_count * 8) ctas = (unsigned)w->sm_count * 8;
    const dsr_u64 t = w->t;
    k_st_f1<L><<<ctas, 256, 0, s>>>(A, w->ws, t);
    k_st_f2<L><<<ctas, 256, 0, s>>>(A, w->ws, t);
    k_st_s0<L><<<ctas, 256, 0, s>>>(A, w->ws);
    k_st_s1<L><<<ctas, 256, 0, s>>>(A, w->ws, t);
    k_st_s2<L><<<ctas, 256, 0, s>>>(A, w->ws, t);
    w->t += 1;
    return dsr__check_launch("dsr_wator_static_step");
}

extern "C" int dsr_wator_static_bytes(int W, int H, int aos, size_t* out) {
    if (!out || W < 3 || H < 3 || (int64_t)W * H >= (1ll << 31)) return DSR_E_INVALID;
    size_t off[6];
    *out = layout(W, H, aos, off);
    return DSR_OK;
}

extern "C" int dsr_wator_static_create(const dsr_wator_params* p, const void* kind0_dev, void* workspace_dev, int aos,
                                       void* stream, dsr_wator_static** out) {
    if (!params_ok(p) || !kind0_dev || !workspace_dev || !out) return DSR_E_INVALID;
    if (reinterpret_cast<uintptr_t>(workspace_dev) & 255) return DSR_E_INVALID;
    size_t off[6];
    layout(p->W, p->H, aos, off);
    uint8_t* base = static_cast<uint8_t*>(workspace_dev);
    dsr_wator_static* w = new dsr_wator_static;
    w->aos = aos ? 1 : 0;
    w->soa = Soa{base + off[0], reinterpret_cast<int32_t*>(base + off[1]), reinterpret_cast<int32_t*>(base + off[2])};
    w->a = Aos{reinterpret_cast<AosCell*>(base + off[0])};
    w->ws = StaticWs{reinterpret_cast<dsr_u64*>(base + off[3]), reinterpret_cast<uint32_t*>(base + off[4]),
                     reinterpret_cast<dsr_u64*>(base + off[5]), *p};
    w->t = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&w->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || w->sm_count < 1)
        w->sm_count = 1;
    cudaStream_t s = dsr__stream(stream);
    cudaError_t e = cudaMemsetAsync(w->ws.visits, 0, 8, s);
    if (e) {
        delete w;
        dsr__set_cuda_error(e, "dsr_wator_static_create");
        return DSR_E_CUDA;
    }
    const uint32_t n = (uint32_t)p->W * (uint32_t)p->H;
    unsigned ctas = (n + 255) / 256;
    if (ctas > (unsigned)w->sm_count * 8) ctas = (unsigned)w->sm_count * 8;
    const uint8_t* k0 = static_cast<const uint8_t*>(kind0_dev);
    if (w->aos)
        k_st_init<Aos><<<ctas, 256, 0, s>>>(w->a, w->ws, k0);
    else
        k_st_init<Soa><<<ctas, 256, 0, s>>>(w->soa, w->ws, k0);
    int rc = dsr__check_launch("dsr_wator_static_create");
    if (rc) {
        delete w;
        return rc;
    }
    *out = w;
    return DSR_OK;
}

extern "C" int dsr_wator_static_step(dsr_wator_static* w, int n_steps, void* stream) {
    if (!w || n_steps < 0) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    for (int i = 0; i < n_steps; ++i) {
        const int rc = w->aos ? launch_step(w, w->a, s) : launch_step(w, w->soa, s);
        if (rc) return rc;
    }
    return DSR_OK;
}

extern "C" int dsr_wator_static_hash(dsr_wator_static* w, void* hash_dev, void* stream) {
    if (!w || !hash_dev) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    const uint32_t n = (uint32_t)w->ws.p.W * (uint32_t)w->ws.p.H;
    unsigned ctas = (n + 255) / 256;
    if (ctas > (unsigned)w->sm_count * 8) ctas = (unsigned)w->sm_count * 8;
    dsr_u64* out = static_cast<dsr_u64*>(hash_dev);
    if (w->aos)
        k_st_hash<Aos><<<ctas, 256, 0, s>>>(w->a, w->ws, out);
    else
        k_st_hash<Soa><<<ctas, 256, 0, s>>>(w->soa, w->ws, out);
    return dsr__check_launch("dsr_wator_static_hash");
}

extern "C" int dsr_wator_static_state(dsr_wator_static* w, void* kind_dev, void* timer_dev, void* energy_dev,
                                      void* stream) {
    if (!w || !kind_dev || !timer_dev || !energy_dev) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    const uint32_t n = (uint32_t)w->ws.p.W * (uint32_t)w->ws.p.H;
    unsigned ctas = (n + 255) / 256;
    if (ctas > (unsigned)w->sm_count * 8) ctas = (unsigned)w->sm_count * 8;
    auto* k = static_cast<uint8_t*>(kind_dev);
    auto* t = static_cast<int32_t*>(timer_dev);
    auto* e = static_cast<int32_t*>(energy_dev);
    if (w->aos)
        k_st_state<Aos><<<ctas, 256, 0, s>>>(w->a, w->ws, k, t, e);
    else
        k_st_state<Soa><<<ctas, 256, 0, s>>>(w->soa, w->ws, k, t, e);
    return dsr__check_launch("dsr_wator_static_state");
}

extern "C" int dsr_wator_static_visits(dsr_wator_static* w, uint64_t* out) {
    if (!w || !out) return DSR_E_INVALID;
    cudaError_t e = cudaMemcpy(out, w->ws.visits, 8, cudaMemcpyDeviceToHost);
    if (e) {
        dsr__set_cuda_error(e, "dsr_wator_static_visits");
        return DSR_E_CUDA;
    }
    return DSR_OK;
}

extern "C" int dsr_wator_static_destroy(dsr_wator_static* w) {
    delete w;
    return DSR_OK;
}
