// Wa-Tor predator-prey as an SMMO program (Fig. 6h): five do-alls per step
// over Fish and Shark objects; births and deaths are device new/delete.
// Rules are stated in dsr_apps.h.
#include "dsr_apps.h"
#include "dsr_internal.cuh"

namespace {
enum { FISH = 0, SHARK = 1 };
enum { X = 0, Y = 1, TIMER = 2, ENERGY = 3 };
enum : dsr_u64 { K_EMPTY = 0, K_FISH = 1, K_SHARK = 2 };
constexpr uint32_t NO_MOVE = 0xFFFFFFFFu;

// Workspace layout (byte offsets); grid and claim are uint64 per cell,
// intent uint32 per cell, then the step counter.
struct WatorWs {
    dsr_u64* grid;    // 0 = empty, else (handle << 2) | kind
    dsr_u64* claim;   // lowest claim key of the current phase
    uint32_t* intent; // target chosen by the agent in this cell, or NO_MOVE
    dsr_u64* step;    // device step counter
};

struct WatorArgs {
    WatorWs ws;
    dsr_wator_params p;
};

// Claim key of phase `ph` (0 fish, 1 shark) of step t for a mover in cell c.
// Keys of later phases compare lower than every key of earlier phases, so the
// claim array never needs resetting; within a phase the lowest cell wins.
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

// F1: age, pick an empty neighbour, claim it.
struct MFishChoose {
    typedef WatorArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        const dsr_u64 t = *(volatile dsr_u64*)a.ws.step;
        const int x = *dsr_field<int32_t>(H, FISH, self, X), y = *dsr_field<int32_t>(H, FISH, self, Y);
        *dsr_field<int32_t>(H, FISH, self, TIMER) += 1;
        const uint32_t c = (uint32_t)(y * a.p.W + x);
        uint32_t nb[4], cand[4];
        neighbours(c, a.p.W, a.p.H, nb);
        int k = 0;
#pragma unroll
        for (int d = 0; d < 4; ++d)
            if (a.ws.grid[nb[d]] == K_EMPTY) cand[k++] = nb[d];
        uint32_t tgt = NO_MOVE;
        if (k) {
            tgt = cand[dsr_rand(a.p.seed, 0, t, c) % (dsr_u64)k];
            atomicMin(a.ws.claim + tgt, claim_key(t, 0, c));
        }
        a.ws.intent[c] = tgt;
    }
};

// F2: winners move and breed.
struct MFishMove {
    typedef WatorArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        const dsr_u64 t = *(volatile dsr_u64*)a.ws.step;
        int32_t* px = dsr_field<int32_t>(H, FISH, self, X);
        int32_t* py = dsr_field<int32_t>(H, FISH, self, Y);
        const uint32_t c = (uint32_t)(*py * a.p.W + *px);
        const uint32_t tgt = a.ws.intent[c];
        if (tgt == NO_MOVE || a.ws.claim[tgt] != claim_key(t, 0, c)) return;
        a.ws.grid[tgt] = (self << 2) | K_FISH;
        *px = (int32_t)(tgt % (uint32_t)a.p.W);
        *py = (int32_t)(tgt / (uint32_t)a.p.W);
        int32_t* timer = dsr_field<int32_t>(H, FISH, self, TIMER);
        dsr_u64 left = K_EMPTY;
        if (*timer >= a.p.fish_breed) {
            *timer = 0;
            const dsr_ref n = dsr_new(H, FISH);
            if (n != DSR_NULL) {
                *dsr_field<int32_t>(H, FISH, n, X) = (int32_t)(c % (uint32_t)a.p.W);
                *dsr_field<int32_t>(H, FISH, n, Y) = (int32_t)(c / (uint32_t)a.p.W);
                *dsr_field<int32_t>(H, FISH, n, TIMER) = 0;
                left = (n << 2) | K_FISH;
            }
        }
        a.ws.grid[c] = left;
    }
};

// S0: starvation.
struct MSharkStarve {
    typedef WatorArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        int32_t* e = dsr_field<int32_t>(H, SHARK, self, ENERGY);
        if (--*e > 0) return;
        const int x = *dsr_field<int32_t>(H, SHARK, self, X), y = *dsr_field<int32_t>(H, SHARK, self, Y);
        a.ws.grid[y * a.p.W + x] = K_EMPTY;
        dsr_delete(H, self);
    }
};

// S1: age, prefer a neighbouring fish, else an empty cell; claim it.
struct MSharkChoose {
    typedef WatorArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        const dsr_u64 t = *(volatile dsr_u64*)a.ws.step;
        const int x = *dsr_field<int32_t>(H, SHARK, self, X), y = *dsr_field<int32_t>(H, SHARK, self, Y);
        *dsr_field<int32_t>(H, SHARK, self, TIMER) += 1;
        const uint32_t c = (uint32_t)(y * a.p.W + x);
        uint32_t nb[4], fish[4], empty[4];
        neighbours(c, a.p.W, a.p.H, nb);
        int kf = 0, ke = 0;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const dsr_u64 g = a.ws.grid[nb[d]];
            if ((g & 3) == K_FISH) fish[kf++] = nb[d];
            else if (g == K_EMPTY) empty[ke++] = nb[d];
        }
        uint32_t tgt = NO_MOVE;
        if (kf || ke) {
            const dsr_u64 r = dsr_rand(a.p.seed, 1, t, c);
            tgt = kf ? fish[r % (dsr_u64)kf] : empty[r % (dsr_u64)ke];
            atomicMin(a.ws.claim + tgt, claim_key(t, 1, c));
        }
        a.ws.intent[c] = tgt;
    }
};

// S2: winners move, eat and breed. The last CTA advances the step counter.
struct MSharkMove {
    typedef WatorArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        const dsr_u64 t = *(volatile dsr_u64*)a.ws.step;
        int32_t* px = dsr_field<int32_t>(H, SHARK, self, X);
        int32_t* py = dsr_field<int32_t>(H, SHARK, self, Y);
        const uint32_t c = (uint32_t)(*py * a.p.W + *px);
        const uint32_t tgt = a.ws.intent[c];
        if (tgt == NO_MOVE || a.ws.claim[tgt] != claim_key(t, 1, c)) return;
        const dsr_u64 g = a.ws.grid[tgt];
        int32_t* energy = dsr_field<int32_t>(H, SHARK, self, ENERGY);
        if ((g & 3) == K_FISH) {
            dsr_delete(H, g >> 2);
            *energy += a.p.shark_gain;
        }
        a.ws.grid[tgt] = (self << 2) | K_SHARK;
        *px = (int32_t)(tgt % (uint32_t)a.p.W);
        *py = (int32_t)(tgt / (uint32_t)a.p.W);
        int32_t* timer = dsr_field<int32_t>(H, SHARK, self, TIMER);
        dsr_u64 left = K_EMPTY;
        if (*timer >= a.p.shark_breed) {
            *timer = 0;
            const dsr_ref n = dsr_new(H, SHARK);
            if (n != DSR_NULL) {
                *dsr_field<int32_t>(H, SHARK, n, X) = (int32_t)(c % (uint32_t)a.p.W);
                *dsr_field<int32_t>(H, SHARK, n, Y) = (int32_t)(c / (uint32_t)a.p.W);
                *dsr_field<int32_t>(H, SHARK, n, TIMER) = 0;
                *dsr_field<int32_t>(H, SHARK, n, ENERGY) = a.p.shark_energy0;
                left = (n << 2) | K_SHARK;
            }
        }
        a.ws.grid[c] = left;
    }
    static __device__ void finish(const dsr_dev_heap&, int, const Args& a) { *a.ws.step += 1; }
};

// One thread per cell: create the initial agents and clear the claim state.
__global__ void k_wator_init(const __grid_constant__ dsr_dev_heap H, const uint8_t* kind0, WatorWs ws,
                             dsr_wator_params p) {
    const uint32_t n = (uint32_t)p.W * (uint32_t)p.H;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const uint8_t k = kind0[c];
        dsr_u64 g = K_EMPTY;
        if (k == 1) {
            const dsr_ref r = dsr_new(H, FISH);
            if (r != DSR_NULL) {
                *dsr_field<int32_t>(H, FISH, r, X) = (int32_t)(c % (uint32_t)p.W);
                *dsr_field<int32_t>(H, FISH, r, Y) = (int32_t)(c / (uint32_t)p.W);
                *dsr_field<int32_t>(H, FISH, r, TIMER) = 0;
                g = (r << 2) | K_FISH;
            }
        } else if (k == 2) {
            const dsr_ref r = dsr_new(H, SHARK);
            if (r != DSR_NULL) {
                *dsr_field<int32_t>(H, SHARK, r, X) = (int32_t)(c % (uint32_t)p.W);
                *dsr_field<int32_t>(H, SHARK, r, Y) = (int32_t)(c / (uint32_t)p.W);
                *dsr_field<int32_t>(H, SHARK, r, TIMER) = 0;
                *dsr_field<int32_t>(H, SHARK, r, ENERGY) = p.shark_energy0;
                g = (r << 2) | K_SHARK;
            }
        }
        ws.grid[c] = g;
        ws.claim[c] = ~0ull;
        ws.intent[c] = NO_MOVE;
        if (c == 0) *ws.step = 0;
    }
}

__global__ void k_wator_kinds(const dsr_u64* grid, uint8_t* out, uint32_t n) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        out[c] = (uint8_t)(grid[c] & 3);
}

const int kFishFields[3] = {4, 4, 4};
const int kSharkFields[4] = {4, 4, 4, 4};

bool heap_matches(const dsr_heap* h) {
    const dsr_layout& L = h->layout;
    if (L.n_types < 2 || L.n_fields[FISH] != 3 || L.n_fields[SHARK] != 4) return false;
    for (int f = 0; f < 3; ++f)
        if (L.field_bytes[FISH][f] != 4) return false;
    for (int f = 0; f < 4; ++f)
        if (L.field_bytes[SHARK][f] != 4) return false;
    return true;
}

size_t ws_bytes(int W, int H) {
    const size_t n = (size_t)W * H;
    return ((n * 8 + 255) / 256 * 256) * 2 + (n * 4 + 255) / 256 * 256 + 256;
}

WatorWs carve(void* base, int W, int H) {
    const size_t n = (size_t)W * H;
    uint8_t* p = static_cast<uint8_t*>(base);
    const size_t g = (n * 8 + 255) / 256 * 256, in = (n * 4 + 255) / 256 * 256;
    WatorWs w;
    w.grid = reinterpret_cast<dsr_u64*>(p);
    w.claim = reinterpret_cast<dsr_u64*>(p + g);
    w.intent = reinterpret_cast<uint32_t*>(p + 2 * g);
    w.step = reinterpret_cast<dsr_u64*>(p + 2 * g + in);
    return w;
}
}  // namespace

struct dsr_wator {
    dsr_heap* heap;
    WatorArgs args;
};

extern "C" int dsr_wator_types(dsr_type_desc* out) {
    if (!out) return DSR_E_INVALID;
    out[0] = dsr_type_desc{"Fish", 3, kFishFields};
    out[1] = dsr_type_desc{"Shark", 4, kSharkFields};
    return DSR_OK;
}

extern "C" int dsr_wator_workspace_bytes(int W, int H, size_t* out) {
    if (!out || W < 3 || H < 3 || (int64_t)W * H >= (1ll << 31)) return DSR_E_INVALID;
    *out = ws_bytes(W, H);
    return DSR_OK;
}

extern "C" int dsr_wator_create(dsr_heap* heap, const dsr_wator_params* p, const void* kind0_dev,
                                void* workspace_dev, void* stream, dsr_wator** out) {
    size_t ws;
    if (!heap || !p || !kind0_dev || !workspace_dev || !out || dsr_wator_workspace_bytes(p->W, p->H, &ws))
        return DSR_E_INVALID;
    if ((reinterpret_cast<uintptr_t>(workspace_dev) & 255) || !heap_matches(heap)) return DSR_E_INVALID;
    if (p->fish_breed < 1 || p->shark_breed < 1 || p->shark_energy0 < 1 || p->shark_gain < 0) return DSR_E_INVALID;
    dsr_wator* w = new dsr_wator;
    w->heap = heap;
    w->args.ws = carve(workspace_dev, p->W, p->H);
    w->args.p = *p;
    const uint32_t n = (uint32_t)p->W * (uint32_t)p->H;
    unsigned ctas = (n + 255) / 256;
    if (ctas > (unsigned)heap->sm_count * 8) ctas = (unsigned)heap->sm_count * 8;
    k_wator_init<<<ctas, 256, 0, dsr__stream(stream)>>>(heap->dev, static_cast<const uint8_t*>(kind0_dev),
                                                         w->args.ws, *p);
    int rc = dsr__check_launch("k_wator_init");
    if (rc) {
        delete w;
        return rc;
    }
    *out = w;
    return DSR_OK;
}

extern "C" int dsr_wator_step(dsr_wator* w, int n_steps, void* stream) {
    if (!w || n_steps < 0) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    dsr_heap* h = w->heap;
    for (int i = 0; i < n_steps; ++i) {
        int rc = dsr__doall<MFishChoose>(h, FISH, w->args, s);
        if (!rc) rc = dsr__doall<MFishMove>(h, FISH, w->args, s);
        if (!rc) rc = dsr__doall<MSharkStarve>(h, SHARK, w->args, s);
        if (!rc) rc = dsr__doall<MSharkChoose>(h, SHARK, w->args, s);
        if (!rc) rc = dsr__doall<MSharkMove>(h, SHARK, w->args, s);
        if (rc) return rc;
    }
    return DSR_OK;
}

extern "C" int dsr_wator_kinds(dsr_wator* w, void* kind_out_dev, void* stream) {
    if (!w || !kind_out_dev) return DSR_E_INVALID;
    const uint32_t n = (uint32_t)w->args.p.W * (uint32_t)w->args.p.H;
    unsigned ctas = (n + 255) / 256;
    if (ctas > (unsigned)w->heap->sm_count * 8) ctas = (unsigned)w->heap->sm_count * 8;
    k_wator_kinds<<<ctas, 256, 0, dsr__stream(stream)>>>(w->args.ws.grid, static_cast<uint8_t*>(kind_out_dev), n);
    return dsr__check_launch("k_wator_kinds");
}

extern "C" int dsr_wator_destroy(dsr_wator* w) {
    delete w;
    return DSR_OK;
}

// dsr_parallel_do entry for the wa-tor phases. Args: a dsr_wator handle
// (pointer-sized), whose workspace and parameters the phase uses.
int dsr__wator_method(dsr_heap* h, int type, int method, const void* args, size_t bytes, cudaStream_t s,
                      bool with_scan) {
    if (!heap_matches(h) || !args || bytes != sizeof(dsr_wator*)) return DSR_E_INVALID;
    dsr_wator* w;
    memcpy(&w, args, sizeof w);
    if (!w || w->heap != h) return DSR_E_INVALID;
    switch (method) {
        case DSR_METHOD_WATOR_F1:
            return type == FISH ? dsr__doall<MFishChoose>(h, type, w->args, s, with_scan) : DSR_E_INVALID;
        case DSR_METHOD_WATOR_F2:
            return type == FISH ? dsr__doall<MFishMove>(h, type, w->args, s, with_scan) : DSR_E_INVALID;
        case DSR_METHOD_WATOR_S0:
            return type == SHARK ? dsr__doall<MSharkStarve>(h, type, w->args, s, with_scan) : DSR_E_INVALID;
        case DSR_METHOD_WATOR_S1:
            return type == SHARK ? dsr__doall<MSharkChoose>(h, type, w->args, s, with_scan) : DSR_E_INVALID;
        case DSR_METHOD_WATOR_S2:
            return type == SHARK ? dsr__doall<MSharkMove>(h, type, w->args, s, with_scan) : DSR_E_INVALID;
        default:
            return DSR_E_INVALID;
    }
}
