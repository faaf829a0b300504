// Wa-Tor predator-prey as an SMMO program (Fig. 6h): five do-alls per step
// over Fish and Shark objects; births and deaths are device new/delete.
// Rules are stated in dsr_apps.h. The rules are written once, over a device
// view of one instance; the plain form runs them as do-alls over one heap,
// the batched form as group do-alls over the heaps of many instances.
#include "dsr_apps.h"
#include "dsr_bitmap_alloc.cuh"
#include "dsr_group.cuh"

namespace {
enum { FISH = 0, SHARK = 1 };
enum { X = 0, Y = 1, TIMER = 2, ENERGY = 3 };
enum : uint32_t { K_EMPTY = 0, K_FISH = 1, K_SHARK = 2 };
constexpr uint32_t NO_MOVE = 0xFFFFFFFFu;
constexpr uint32_t NO_CLAIM = 0xFFFFFFFFu;  // a claim word no mover holds (cells are below 2^31)

// Device view of one instance: its workspace and its parameters.
struct WatorInst {
    uint32_t* grid;    // 0 = empty, else (compact handle << 2) | kind (grid_word)
    uint32_t* claim;   // the lowest mover cell that claimed the cell this phase, or NO_CLAIM
    uint32_t* intent;  // per object slot (intent_index): its chosen target, or NO_MOVE
    dsr_u64 n_slots;   // entries of intent
    dsr_u64* step;     // device step counter (nullptr: unused batch slot)
    dsr_wator_params p;
};

// Grid words are 32 bits: the kind in the low two bits and a compact handle
// above them. dsr heap: the handle itself (block * 64 + slot, below 2^30
// for heaps of at most 2^24 blocks); BitmapAlloc: the slot in the type's
// array (below 2^30), the type following from the kind.
__device__ __forceinline__ uint32_t grid_word(const dsr_dev_heap&, dsr_ref r, uint32_t kind) {
    return ((uint32_t)r << 2) | kind;
}
__device__ __forceinline__ dsr_ref grid_ref(const dsr_dev_heap&, uint32_t g) { return g >> 2; }
__device__ __forceinline__ uint32_t grid_word(const dsr_bm_dev&, dsr_ref r, uint32_t kind) {
    return ((uint32_t)(r & ((1ull << DSR_BM_SLOT_BITS) - 1)) << 2) | kind;
}
__device__ __forceinline__ dsr_ref grid_ref(const dsr_bm_dev&, uint32_t g) {
    const dsr_u64 type = (g & 3) == K_FISH ? 0 : 1;  // Fish = 0, Shark = 1
    return (type << DSR_BM_SLOT_BITS) | (g >> 2);
}

// Intents are indexed by the object's slot, not by its cell: the move phase
// then reads its own intent together with its fields (one round trip), and
// the choose phase writes them coalesced. dsr heap: handle = block * 64 +
// slot; BitmapAlloc: the slot of the type's array.
__device__ __forceinline__ dsr_u64 intent_index(const dsr_dev_heap&, dsr_ref r) { return r; }
__device__ __forceinline__ dsr_u64 intent_index(const dsr_bm_dev&, dsr_ref r) {
    return r & ((1ull << DSR_BM_SLOT_BITS) - 1);
}

// Claims: a mover in cell c claims its target with atomicMin(claim, c), so
// the lowest mover cell wins a contested cell. The winner's move phase puts
// the word back to NO_CLAIM once it has read it; a loser that reads the
// word afterwards sees NO_CLAIM, which is no cell, and loses all the same.
// Every claimed cell has a winner (no mover dies between its choose and move
// phases), so every word is NO_CLAIM again when a choose phase starts.

__device__ __forceinline__ void neighbours(uint32_t c, int W, int H, uint32_t nb[4]) {
    const int x = (int)(c % (uint32_t)W), y = (int)(c / (uint32_t)W);
    nb[0] = (uint32_t)((y == 0 ? H - 1 : y - 1) * W + x);  // N
    nb[1] = (uint32_t)(y * W + (x == W - 1 ? 0 : x + 1));  // E
    nb[2] = (uint32_t)((y == H - 1 ? 0 : y + 1) * W + x);  // S
    nb[3] = (uint32_t)(y * W + (x == 0 ? W - 1 : x - 1));  // W
}

// Checked builds only: the instance exists and c is one of its cells.
template <class HP>
__device__ __forceinline__ bool cell_ok(const HP& H, const WatorInst& I, uint32_t c, unsigned code) {
    return dsr_check(I.grid != nullptr && c < (uint32_t)I.p.W * (uint32_t)I.p.H, H.err, H.dbg, code, c);
}

// The k-th (0-based) set position among the low 4 bits of m, as a neighbour index.
__device__ __forceinline__ int pick(unsigned m, unsigned k) {
    for (int d = 0; d < 4; ++d)
        if ((m >> d) & 1u) {
            if (k == 0) return d;
            --k;
        }
    return 0;
}

// F1: age, pick an empty neighbour, claim it.
template <class HP>
__device__ __forceinline__ void fish_choose(const HP& H, const WatorInst& I, dsr_ref self) {
    const dsr_u64 t = *(volatile dsr_u64*)I.step;
    const int x = *dsr_field<int32_t>(H, FISH, self, X), y = *dsr_field<int32_t>(H, FISH, self, Y);
    *dsr_field<int32_t>(H, FISH, self, TIMER) += 1;
    const uint32_t c = (uint32_t)(y * I.p.W + x);
    if (!cell_ok(H, I, c, 6)) return;
    uint32_t nb[4];
    neighbours(c, I.p.W, I.p.H, nb);
    unsigned m = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) m |= (I.grid[nb[d]] == K_EMPTY ? 1u : 0u) << d;
    uint32_t tgt = NO_MOVE;
    if (m) {
        tgt = nb[pick(m, (unsigned)(dsr_rand(I.p.seed, 0, t, c) % (dsr_u64)__popc(m)))];
        atomicMin(I.claim + tgt, c);
    }
    const dsr_u64 ix = intent_index(H, self);
    if (dsr_check(ix < I.n_slots, H.err, H.dbg, 8, ix)) I.intent[ix] = tgt;
}

// F2: winners move and breed.
template <class HP>
__device__ __forceinline__ void fish_move(const HP& H, const WatorInst& I, dsr_ref self) {
    int32_t* px = dsr_field<int32_t>(H, FISH, self, X);
    int32_t* py = dsr_field<int32_t>(H, FISH, self, Y);
    int32_t* timer = dsr_field<int32_t>(H, FISH, self, TIMER);
    const dsr_u64 ix = intent_index(H, self);
    if (!dsr_check(ix < I.n_slots, H.err, H.dbg, 8, ix)) return;
    // timer and intent are loaded with x and y: one round trip for all four
    const int32_t age = *timer;
    const uint32_t tgt = I.intent[ix];
    const uint32_t c = (uint32_t)(*py * I.p.W + *px);
    if (!cell_ok(H, I, c, 6)) return;
    if (tgt != NO_MOVE && !cell_ok(H, I, tgt, 7)) return;
    if (tgt == NO_MOVE || I.claim[tgt] != c) return;
    I.claim[tgt] = NO_CLAIM;
    dsr_count_lanes(H.ctr, DSR_CTR_APP0);
    I.grid[tgt] = grid_word(H, self, K_FISH);
    *px = (int32_t)(tgt % (uint32_t)I.p.W);
    *py = (int32_t)(tgt / (uint32_t)I.p.W);
    uint32_t left = K_EMPTY;
    if (age >= I.p.fish_breed) {
        *timer = 0;
        const dsr_ref n = dsr_new(H, FISH);
        if (n != DSR_NULL) {
            *dsr_field<int32_t>(H, FISH, n, X) = (int32_t)(c % (uint32_t)I.p.W);
            *dsr_field<int32_t>(H, FISH, n, Y) = (int32_t)(c / (uint32_t)I.p.W);
            *dsr_field<int32_t>(H, FISH, n, TIMER) = 0;
            left = grid_word(H, n, K_FISH);
        }
    }
    I.grid[c] = left;
}

// S0: starvation.
template <class HP>
__device__ __forceinline__ void shark_starve(const HP& H, const WatorInst& I, dsr_ref self) {
    int32_t* e = dsr_field<int32_t>(H, SHARK, self, ENERGY);
    if (--*e > 0) return;
    const int x = *dsr_field<int32_t>(H, SHARK, self, X), y = *dsr_field<int32_t>(H, SHARK, self, Y);
    if (cell_ok(H, I, (uint32_t)(y * I.p.W + x), 6)) I.grid[y * I.p.W + x] = K_EMPTY;
    dsr_delete(H, self);
}

// S1: age, prefer a neighbouring fish, else an empty cell; claim it.
template <class HP>
__device__ __forceinline__ void shark_choose(const HP& H, const WatorInst& I, dsr_ref self) {
    const dsr_u64 t = *(volatile dsr_u64*)I.step;
    const int x = *dsr_field<int32_t>(H, SHARK, self, X), y = *dsr_field<int32_t>(H, SHARK, self, Y);
    *dsr_field<int32_t>(H, SHARK, self, TIMER) += 1;
    const uint32_t c = (uint32_t)(y * I.p.W + x);
    if (!cell_ok(H, I, c, 6)) return;
    uint32_t nb[4];
    neighbours(c, I.p.W, I.p.H, nb);
    unsigned mf = 0, me = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const uint32_t g = I.grid[nb[d]];
        mf |= ((g & 3) == K_FISH ? 1u : 0u) << d;
        me |= (g == K_EMPTY ? 1u : 0u) << d;
    }
    const unsigned m = mf ? mf : me;
    uint32_t tgt = NO_MOVE;
    if (m) {
        tgt = nb[pick(m, (unsigned)(dsr_rand(I.p.seed, 1, t, c) % (dsr_u64)__popc(m)))];
        atomicMin(I.claim + tgt, c);
    }
    const dsr_u64 ix = intent_index(H, self);
    if (dsr_check(ix < I.n_slots, H.err, H.dbg, 8, ix)) I.intent[ix] = tgt;
}

// S2: winners move, eat and breed.
template <class HP>
__device__ __forceinline__ void shark_move(const HP& H, const WatorInst& I, dsr_ref self) {
    int32_t* px = dsr_field<int32_t>(H, SHARK, self, X);
    int32_t* py = dsr_field<int32_t>(H, SHARK, self, Y);
    int32_t* timer = dsr_field<int32_t>(H, SHARK, self, TIMER);
    int32_t* energy = dsr_field<int32_t>(H, SHARK, self, ENERGY);
    const dsr_u64 ix = intent_index(H, self);
    if (!dsr_check(ix < I.n_slots, H.err, H.dbg, 8, ix)) return;
    const int32_t age = *timer, e0 = *energy;  // loaded with x and y
    const uint32_t tgt = I.intent[ix];
    const uint32_t c = (uint32_t)(*py * I.p.W + *px);
    if (!cell_ok(H, I, c, 6)) return;
    if (tgt != NO_MOVE && !cell_ok(H, I, tgt, 7)) return;
    if (tgt == NO_MOVE || I.claim[tgt] != c) return;
    I.claim[tgt] = NO_CLAIM;
    dsr_count_lanes(H.ctr, DSR_CTR_APP0);
    const uint32_t g = I.grid[tgt];
    if ((g & 3) == K_FISH) {
        dsr_delete(H, grid_ref(H, g));
        *energy = e0 + I.p.shark_gain;
    }
    I.grid[tgt] = grid_word(H, self, K_SHARK);
    *px = (int32_t)(tgt % (uint32_t)I.p.W);
    *py = (int32_t)(tgt / (uint32_t)I.p.W);
    uint32_t left = K_EMPTY;
    if (age >= I.p.shark_breed) {
        *timer = 0;
        const dsr_ref n = dsr_new(H, SHARK);
        if (n != DSR_NULL) {
            *dsr_field<int32_t>(H, SHARK, n, X) = (int32_t)(c % (uint32_t)I.p.W);
            *dsr_field<int32_t>(H, SHARK, n, Y) = (int32_t)(c / (uint32_t)I.p.W);
            *dsr_field<int32_t>(H, SHARK, n, TIMER) = 0;
            *dsr_field<int32_t>(H, SHARK, n, ENERGY) = I.p.shark_energy0;
            left = grid_word(H, n, K_SHARK);
        }
    }
    I.grid[c] = left;
}

// ---- plain form: do-all methods over one heap ------------------------------
// (HP: the heap type; dsr_dev_heap, or dsr_bm_dev for the BitmapAlloc
// comparator)
template <class HP>
struct MFishChooseT {
    typedef WatorInst Args;
    static __device__ void run(const HP& H, int, const Args& a, dsr_ref s) { fish_choose(H, a, s); }
};
template <class HP>
struct MFishMoveT {
    typedef WatorInst Args;
    static __device__ void run(const HP& H, int, const Args& a, dsr_ref s) { fish_move(H, a, s); }
};
template <class HP>
struct MSharkStarveT {
    typedef WatorInst Args;
    static __device__ void run(const HP& H, int, const Args& a, dsr_ref s) { shark_starve(H, a, s); }
};
template <class HP>
struct MSharkChooseT {
    typedef WatorInst Args;
    static __device__ void run(const HP& H, int, const Args& a, dsr_ref s) { shark_choose(H, a, s); }
};
// The last CTA of the last phase advances the step counter.
template <class HP>
struct MSharkMoveT {
    typedef WatorInst Args;
    static __device__ void run(const HP& H, int, const Args& a, dsr_ref s) { shark_move(H, a, s); }
    static __device__ void finish(const HP&, int, const Args& a) { *a.step += 1; }
};
typedef MFishChooseT<dsr_dev_heap> MFishChoose;
typedef MFishMoveT<dsr_dev_heap> MFishMove;
typedef MSharkStarveT<dsr_dev_heap> MSharkStarve;
typedef MSharkChooseT<dsr_dev_heap> MSharkChoose;
typedef MSharkMoveT<dsr_dev_heap> MSharkMove;

// ---- batched form: group do-all methods over the heaps of many instances ----
// Heap index h of a group is the instance slot; table[h] is its view.
struct BatchArgs {
    const WatorInst* table;
};
struct GFishChoose {
    typedef BatchArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref s, uint32_t h) {
        fish_choose(H, a.table[h], s);
    }
};
struct GFishMove {
    typedef BatchArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref s, uint32_t h) {
        fish_move(H, a.table[h], s);
    }
};
struct GSharkStarve {
    typedef BatchArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref s, uint32_t h) {
        shark_starve(H, a.table[h], s);
    }
};
struct GSharkChoose {
    typedef BatchArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref s, uint32_t h) {
        shark_choose(H, a.table[h], s);
    }
};
struct GSharkMove {
    typedef BatchArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref s, uint32_t h) {
        shark_move(H, a.table[h], s);
    }
    // every instance in the batch advances one step
    static __device__ void finish_group(const dsr_group_dev& G, int, const Args& a) {
        for (uint32_t i = threadIdx.x; i < G.n_slots; i += blockDim.x)
            if (a.table[i].step) *a.table[i].step += 1;
    }
};

// One thread per cell: create the initial agents and clear the claim state.
template <class HP>
__global__ void k_wator_init(const __grid_constant__ HP H, const uint8_t* kind0, WatorInst I) {
    const uint32_t n = (uint32_t)I.p.W * (uint32_t)I.p.H;
    const uint32_t n32 = (n + 31u) & ~31u;  // warp-uniform trip count
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n32; c += gridDim.x * blockDim.x) {
        __syncwarp();  // whole-warp groups for dsr_new
        if (c >= n) continue;
        const uint8_t k = kind0[c];
        uint32_t g = K_EMPTY;
        if (k == 1 || k == 2) {
            // one dsr_new for fish and sharks: the two groups' leaders then
            // run their reservations side by side rather than one after the
            // other in two branches
            const int T = k == 1 ? FISH : SHARK;
            const dsr_ref r = dsr_new(H, T);
            if (r != DSR_NULL) {
                *dsr_field<int32_t>(H, T, r, X) = (int32_t)(c % (uint32_t)I.p.W);
                *dsr_field<int32_t>(H, T, r, Y) = (int32_t)(c / (uint32_t)I.p.W);
                *dsr_field<int32_t>(H, T, r, TIMER) = 0;
                if (T == SHARK) *dsr_field<int32_t>(H, SHARK, r, ENERGY) = I.p.shark_energy0;
                g = grid_word(H, r, k == 1 ? K_FISH : K_SHARK);
            }
        }
        I.grid[c] = g;
        I.claim[c] = NO_CLAIM;
        if (c == 0) *I.step = 0;
    }
}

__global__ void k_wator_kinds(const uint32_t* grid, uint8_t* out, uint32_t n) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        out[c] = (uint8_t)(grid[c] & 3);
}

const int kFishFields[3] = {4, 4, 4};
const int kSharkFields[4] = {4, 4, 4, 4};

// Grid words hold handles below 2^30: heaps of at most 2^24 blocks.
constexpr dsr_u64 kMaxBlocks = 1ull << 24;

bool heap_matches(const dsr_heap* h) {
    const dsr_layout& L = h->layout;
    if (L.n_blocks > kMaxBlocks) return false;
    if (L.n_types < 2 || L.n_fields[FISH] != 3 || L.n_fields[SHARK] != 4) return false;
    for (int f = 0; f < 3; ++f)
        if (L.field_bytes[FISH][f] != 4) return false;
    for (int f = 0; f < 4; ++f)
        if (L.field_bytes[SHARK][f] != 4) return false;
    return true;
}

bool params_ok(const dsr_wator_params* p) {
    return p && p->W >= 3 && p->H >= 3 && (int64_t)p->W * p->H < (1ll << 31) && p->fish_breed >= 1 &&
           p->shark_breed >= 1 && p->shark_energy0 >= 1 && p->shark_gain >= 0;
}

// Workspace: grid u32[n] | claim u32[n] | step counter (256 B) | intent
// u32[slots], each part 256-byte aligned; slots = object slots of the heap.
size_t ws_bytes(int W, int H, dsr_u64 slots) {
    const size_t n = (size_t)W * H;
    return ((n * 4 + 255) / 256 * 256) * 2 + 256 + (slots * 4 + 255) / 256 * 256;
}

WatorInst carve(void* base, const dsr_wator_params& p, dsr_u64 slots) {
    const size_t n = (size_t)p.W * p.H;
    uint8_t* b = static_cast<uint8_t*>(base);
    const size_t g = (n * 4 + 255) / 256 * 256;
    WatorInst w;
    w.grid = reinterpret_cast<uint32_t*>(b);
    w.claim = reinterpret_cast<uint32_t*>(b + g);
    w.step = reinterpret_cast<dsr_u64*>(b + 2 * g);
    w.intent = reinterpret_cast<uint32_t*>(b + 2 * g + 256);
    w.n_slots = slots;
    w.p = p;
    return w;
}

dsr_u64 heap_slots(const dsr_heap* h) { return h->layout.n_blocks * 64; }
dsr_u64 bm_slots(const dsr_bm_heap* h) {
    return h->dev.cap[FISH] > h->dev.cap[SHARK] ? h->dev.cap[FISH] : h->dev.cap[SHARK];
}

int launch_init(const dsr_heap* heap, const WatorInst& I, const void* kind0_dev, cudaStream_t s) {
    const uint32_t n = (uint32_t)I.p.W * (uint32_t)I.p.H;
    unsigned ctas = (n + 255) / 256;
    if (ctas > (unsigned)heap->sm_count * 8) ctas = (unsigned)heap->sm_count * 8;
    k_wator_init<dsr_dev_heap><<<ctas, 256, 0, s>>>(heap->dev, static_cast<const uint8_t*>(kind0_dev), I);
    return dsr__check_launch("k_wator_init");
}

int launch_kinds(const dsr_heap* heap, const WatorInst& I, void* out, cudaStream_t s) {
    const uint32_t n = (uint32_t)I.p.W * (uint32_t)I.p.H;
    unsigned ctas = (n + 255) / 256;
    if (ctas > (unsigned)heap->sm_count * 8) ctas = (unsigned)heap->sm_count * 8;
    k_wator_kinds<<<ctas, 256, 0, s>>>(I.grid, static_cast<uint8_t*>(out), n);
    return dsr__check_launch("k_wator_kinds");
}
}  // namespace

// ===========================================================================
// plain form
// ===========================================================================
constexpr int kPhaseEvents = 11;  // step start, then after each scan and each method kernel

// One step replayed as a CUDA graph: its 8 launches (and, when the step is
// timed, its event records as event-record nodes, pointed at each step's
// own events before the launch). Captured on first use, once for untimed
// steps and once for the current timing selection.
struct StepGraph {
    cudaGraph_t graph = nullptr;  // kept while exec lives: ev_node are its nodes
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t ev_node[kPhaseEvents] = {};  // timed graph: the node of event k, or null
    int sel = -2;                                // timing selection captured (-2: untimed)
    uint64_t version = 0;                        // the heap view's version captured
};

struct dsr_wator {
    dsr_heap* heap;
    WatorInst inst;
    // phase timing: kPhaseEvents events per step, created when enabled
    std::vector<cudaEvent_t> ev;
    int ev_steps = 0;  // steps recorded in the current window
    int ev_phase = -1; // the one phase whose method kernel is timed, or -1: all
    StepGraph plain, timed;
    cudaStream_t capture = nullptr;  // private stream for the captures
    bool graphs_off = false;         // a capture failed: launch kernel by kernel
};

static void drop_graph(StepGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g = StepGraph{};
}

static void free_events(dsr_wator* w) {
    drop_graph(w->timed);  // its nodes name these events
    for (cudaEvent_t e : w->ev) cudaEventDestroy(e);
    w->ev.clear();
    w->ev_steps = 0;
}

extern "C" int dsr_wator_types(dsr_type_desc* out) {
    if (!out) return DSR_E_INVALID;
    out[0] = dsr_type_desc{"Fish", 3, kFishFields};
    out[1] = dsr_type_desc{"Shark", 4, kSharkFields};
    return DSR_OK;
}

extern "C" int dsr_wator_workspace_bytes(const dsr_heap* heap, int W, int H, size_t* out) {
    if (!heap || !out || W < 3 || H < 3 || (int64_t)W * H >= (1ll << 31)) return DSR_E_INVALID;
    *out = ws_bytes(W, H, heap_slots(heap));
    return DSR_OK;
}

extern "C" int dsr_wator_bm_workspace_bytes(const dsr_bm_heap* heap, int W, int H, size_t* out) {
    if (!heap || !out || W < 3 || H < 3 || (int64_t)W * H >= (1ll << 31)) return DSR_E_INVALID;
    *out = ws_bytes(W, H, bm_slots(heap));
    return DSR_OK;
}

extern "C" int dsr_wator_create(dsr_heap* heap, const dsr_wator_params* p, const void* kind0_dev,
                                void* workspace_dev, void* stream, dsr_wator** out) {
    if (!heap || !params_ok(p) || !kind0_dev || !workspace_dev || !out) return DSR_E_INVALID;
    if ((reinterpret_cast<uintptr_t>(workspace_dev) & 255) || !heap_matches(heap)) return DSR_E_INVALID;
    dsr_wator* w = new dsr_wator;
    w->heap = heap;
    w->inst = carve(workspace_dev, *p, heap_slots(heap));
    int rc = launch_init(heap, w->inst, kind0_dev, dsr__stream(stream));
    if (rc) {
        delete w;
        return rc;
    }
    *out = w;
    return DSR_OK;
}

extern "C" int dsr_wator_attach(dsr_heap* heap, const dsr_wator_params* p, void* workspace_dev, dsr_wator** out) {
    if (!heap || !params_ok(p) || !workspace_dev || !out) return DSR_E_INVALID;
    if ((reinterpret_cast<uintptr_t>(workspace_dev) & 255) || !heap_matches(heap)) return DSR_E_INVALID;
    dsr_wator* w = new dsr_wator;
    w->heap = heap;
    w->inst = carve(workspace_dev, *p, heap_slots(heap));
    *out = w;
    return DSR_OK;
}

// The launches of one step on s; e: the step's kPhaseEvents events (null:
// untimed), of which only the selected phase's two are recorded when sel >= 0.
static int issue_step(dsr_wator* w, cudaStream_t s, const cudaEvent_t* e, int sel) {
    dsr_heap* h = w->heap;
    if (e && sel < 0) cudaEventRecordWithFlags(e[0], s, cudaEventRecordExternal);
    // event k: k = 2p + 1 after phase p's scan, k = 2p + 2 after its method
    auto E = [&](int k) -> cudaEvent_t {
        if (!e || (sel >= 0 && k != 2 * sel + 1 && k != 2 * sel + 2)) return nullptr;
        return e[k];
    };
    // F1 neither creates nor deletes fish, so F2 runs over F1's block list
    // (the fish live at the start of the step); likewise S2 over S1's (the
    // sharks that survived S0).
    int rc = dsr__doall<MFishChoose>(h, FISH, w->inst, s, true, E(1), E(2), 1);
    if (!rc) rc = dsr__doall<MFishMove>(h, FISH, w->inst, s, false, E(3), E(4));
    if (!rc) rc = dsr__doall<MSharkStarve>(h, SHARK, w->inst, s, true, E(5), E(6));
    if (!rc) rc = dsr__doall<MSharkChoose>(h, SHARK, w->inst, s, true, E(7), E(8), 1);
    if (!rc) rc = dsr__doall<MSharkMove>(h, SHARK, w->inst, s, false, E(9), E(10));
    return rc;
}

// Capture one step into g (timed with the events e as placeholders when e is
// given). Returns false, leaving g empty, if any step of it fails.
static bool capture_step(dsr_wator* w, StepGraph& g, const cudaEvent_t* e, int sel) {
    if (!w->capture && cudaStreamCreateWithFlags(&w->capture, cudaStreamNonBlocking) != cudaSuccess) {
        w->capture = nullptr;
        return false;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(w->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    const int rc = issue_step(w, w->capture, e, sel);
    const cudaError_t end = cudaStreamEndCapture(w->capture, &graph);
    bool ok = rc == DSR_OK && end == cudaSuccess && graph;
    StepGraph out;
    out.sel = e ? sel : -2;
    out.version = w->heap->version;
    if (ok && e) {
        // the event-record nodes, by the placeholder event they record
        size_t n = 0;
        ok = cudaGraphGetNodes(graph, nullptr, &n) == cudaSuccess;
        std::vector<cudaGraphNode_t> nodes(n);
        if (ok && n) ok = cudaGraphGetNodes(graph, nodes.data(), &n) == cudaSuccess;
        for (size_t i = 0; ok && i < n; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess) ok = false;
            if (!ok || t != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev = nullptr;
            if (cudaGraphEventRecordNodeGetEvent(nodes[i], &ev) != cudaSuccess) ok = false;
            for (int k = 0; ok && k < kPhaseEvents; ++k)
                if (ev == e[k]) out.ev_node[k] = nodes[i];
        }
    }
    if (ok) ok = cudaGraphInstantiate(&out.exec, graph, 0) == cudaSuccess;
    out.graph = graph;
    cudaGetLastError();  // a failed capture leaves no error behind for later calls
    if (!ok) {
        drop_graph(out);
        return false;
    }
    drop_graph(g);
    g = out;
    return true;
}

// Capture the timed step graph for the current selection now, with the
// window's first events as placeholders, so that a timed step does not
// spend its time in a capture.
static void prepare_timed(dsr_wator* w) {
    if (w->graphs_off || w->ev.empty()) return;
    if (!capture_step(w, w->timed, w->ev.data(), w->ev_phase)) w->graphs_off = true;
}

// One step by graph replay; false if the graph cannot be had (the caller
// then launches the step kernel by kernel).
static bool replay_step(dsr_wator* w, cudaStream_t s, const cudaEvent_t* e, int sel, int* rc) {
    StepGraph& g = e ? w->timed : w->plain;
    if (!g.exec || (e && g.sel != sel) || g.version != w->heap->version) {
        if (!capture_step(w, g, e, sel)) return false;
    }
    cudaError_t err = cudaSuccess;
    if (e)
        for (int k = 0; k < kPhaseEvents && err == cudaSuccess; ++k)
            if (g.ev_node[k]) err = cudaGraphExecEventRecordNodeSetEvent(g.exec, g.ev_node[k], e[k]);
    if (err != cudaSuccess) {  // nothing launched yet: the caller launches the step itself
        cudaGetLastError();
        return false;
    }
    err = cudaGraphLaunch(g.exec, s);
    if (err != cudaSuccess) {
        dsr__set_cuda_error(err, "dsr_wator_step graph");
        *rc = DSR_E_CUDA;
    } else {
        *rc = DSR_OK;
    }
    return true;
}

extern "C" int dsr_wator_step(dsr_wator* w, int n_steps, void* stream) {
    if (!w || n_steps < 0) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    // Steps are replayed as a captured graph, except while the caller's
    // stream is itself being captured (the kernels then go into the caller's
    // graph) or after a capture failed.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool use_graph = !w->graphs_off && cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
                           cs == cudaStreamCaptureStatusNone;
    for (int i = 0; i < n_steps; ++i) {
        cudaEvent_t* e = nullptr;
        if ((size_t)(w->ev_steps + 1) * kPhaseEvents <= w->ev.size())
            e = w->ev.data() + (size_t)w->ev_steps++ * kPhaseEvents;
        int rc = DSR_OK;
        if (use_graph && !w->graphs_off) {
            if (replay_step(w, s, e, w->ev_phase, &rc)) {
                if (rc) return rc;
                continue;
            }
            w->graphs_off = true;
        }
        rc = issue_step(w, s, e, w->ev_phase);
        if (rc) return rc;
    }
    return DSR_OK;
}

extern "C" int dsr_wator_phase_timing(dsr_wator* w, int max_steps) {
    if (!w || max_steps < 0) return DSR_E_INVALID;
    free_events(w);
    for (size_t k = 0; k < (size_t)max_steps * kPhaseEvents; ++k) {
        cudaEvent_t e;
        const cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) {
            free_events(w);
            dsr__set_cuda_error(err, "cudaEventCreate");
            return DSR_E_CUDA;
        }
        w->ev.push_back(e);
    }
    prepare_timed(w);
    return DSR_OK;
}

extern "C" int dsr_wator_phase_select(dsr_wator* w, int phase) {
    if (!w || phase < -1 || phase > 4) return DSR_E_INVALID;
    w->ev_phase = phase;
    w->ev_steps = 0;  // a window records one selection
    drop_graph(w->timed);
    prepare_timed(w);
    return DSR_OK;
}

extern "C" int dsr_wator_phase_times(dsr_wator* w, double* out_ms, int* steps) {
    if (!w || !out_ms || !steps) return DSR_E_INVALID;
    for (int k = 0; k < 10; ++k) out_ms[k] = 0;
    *steps = w->ev_steps;
    const int sel = w->ev_phase;
    if (w->ev_steps && sel >= 0) {
        // only the selected phase's method kernel was bracketed
        const size_t last = (size_t)(w->ev_steps - 1) * kPhaseEvents + 2 * sel + 2;
        cudaError_t err = cudaEventSynchronize(w->ev[last]);
        for (int i = 0; i < w->ev_steps && err == cudaSuccess; ++i) {
            const cudaEvent_t* e = w->ev.data() + (size_t)i * kPhaseEvents;
            float run = 0;
            err = cudaEventElapsedTime(&run, e[2 * sel + 1], e[2 * sel + 2]);
            out_ms[sel] += run;
        }
        if (err != cudaSuccess) {
            dsr__set_cuda_error(err, "dsr_wator_phase_times");
            return DSR_E_CUDA;
        }
    } else if (w->ev_steps) {
        cudaError_t err = cudaEventSynchronize(w->ev[(size_t)w->ev_steps * kPhaseEvents - 1]);
        for (int i = 0; i < w->ev_steps && err == cudaSuccess; ++i) {
            const cudaEvent_t* e = w->ev.data() + (size_t)i * kPhaseEvents;
            for (int p = 0; p < 5 && err == cudaSuccess; ++p) {
                float scan = 0, run = 0;
                err = cudaEventElapsedTime(&scan, e[2 * p], e[2 * p + 1]);
                if (err == cudaSuccess) err = cudaEventElapsedTime(&run, e[2 * p + 1], e[2 * p + 2]);
                out_ms[p] += run;
                out_ms[5 + p] += scan;
            }
        }
        if (err != cudaSuccess) {
            dsr__set_cuda_error(err, "dsr_wator_phase_times");
            return DSR_E_CUDA;
        }
    }
    w->ev_steps = 0;
    return DSR_OK;
}

extern "C" int dsr_wator_kinds(dsr_wator* w, void* kind_out_dev, void* stream) {
    if (!w || !kind_out_dev) return DSR_E_INVALID;
    return launch_kinds(w->heap, w->inst, kind_out_dev, dsr__stream(stream));
}

extern "C" int dsr_wator_destroy(dsr_wator* w) {
    if (w) {
        free_events(w);
        drop_graph(w->plain);
        if (w->capture) cudaStreamDestroy(w->capture);
    }
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
            return type == FISH ? dsr__doall<MFishChoose>(h, type, w->inst, s, with_scan) : DSR_E_INVALID;
        case DSR_METHOD_WATOR_F2:
            return type == FISH ? dsr__doall<MFishMove>(h, type, w->inst, s, with_scan) : DSR_E_INVALID;
        case DSR_METHOD_WATOR_S0:
            return type == SHARK ? dsr__doall<MSharkStarve>(h, type, w->inst, s, with_scan) : DSR_E_INVALID;
        case DSR_METHOD_WATOR_S1:
            return type == SHARK ? dsr__doall<MSharkChoose>(h, type, w->inst, s, with_scan) : DSR_E_INVALID;
        case DSR_METHOD_WATOR_S2:
            return type == SHARK ? dsr__doall<MSharkMove>(h, type, w->inst, s, with_scan) : DSR_E_INVALID;
        default:
            return DSR_E_INVALID;
    }
}

// ===========================================================================
// the same rules on the BitmapAlloc comparator (dsr_bitmap_alloc.cuh)
// ===========================================================================
struct dsr_wator_bm {
    dsr_bm_heap* heap;
    WatorInst inst;
};

static bool bm_heap_matches(const dsr_bm_heap* h) {
    if (bm_slots(h) > (1ull << 30)) return false;  // grid words hold slots below 2^30
    if (h->n_types < 2 || h->n_fields[FISH] != 3 || h->n_fields[SHARK] != 4) return false;
    for (int f = 0; f < 3; ++f)
        if (h->field_bytes[FISH][f] != 4) return false;
    for (int f = 0; f < 4; ++f)
        if (h->field_bytes[SHARK][f] != 4) return false;
    return true;
}

extern "C" int dsr_wator_bm_create(dsr_bm_heap* heap, const dsr_wator_params* p, const void* kind0_dev,
                                   void* workspace_dev, void* stream, dsr_wator_bm** out) {
    if (!heap || !params_ok(p) || !kind0_dev || !workspace_dev || !out) return DSR_E_INVALID;
    if ((reinterpret_cast<uintptr_t>(workspace_dev) & 255) || !bm_heap_matches(heap)) return DSR_E_INVALID;
    dsr_wator_bm* w = new dsr_wator_bm;
    w->heap = heap;
    w->inst = carve(workspace_dev, *p, bm_slots(heap));
    const uint32_t n = (uint32_t)p->W * (uint32_t)p->H;
    unsigned ctas = (n + 255) / 256;
    if (ctas > (unsigned)heap->sm_count * 8) ctas = (unsigned)heap->sm_count * 8;
    k_wator_init<dsr_bm_dev>
        <<<ctas, 256, 0, dsr__stream(stream)>>>(heap->dev, static_cast<const uint8_t*>(kind0_dev), w->inst);
    const int rc = dsr__check_launch("k_wator_init");
    if (rc) {
        delete w;
        return rc;
    }
    *out = w;
    return DSR_OK;
}

extern "C" int dsr_wator_bm_step(dsr_wator_bm* w, int n_steps, void* stream) {
    if (!w || n_steps < 0) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    dsr_bm_heap* h = w->heap;
    for (int i = 0; i < n_steps; ++i) {
        // list reuse for F2 and S2 as in dsr_wator_step
        int rc = dsr__bm_doall<MFishChooseT<dsr_bm_dev>>(h, FISH, w->inst, s, true, 1);
        if (!rc) rc = dsr__bm_doall<MFishMoveT<dsr_bm_dev>>(h, FISH, w->inst, s, false);
        if (!rc) rc = dsr__bm_doall<MSharkStarveT<dsr_bm_dev>>(h, SHARK, w->inst, s);
        if (!rc) rc = dsr__bm_doall<MSharkChooseT<dsr_bm_dev>>(h, SHARK, w->inst, s, true, 1);
        if (!rc) rc = dsr__bm_doall<MSharkMoveT<dsr_bm_dev>>(h, SHARK, w->inst, s, false);
        if (rc) return rc;
    }
    return DSR_OK;
}

extern "C" int dsr_wator_bm_destroy(dsr_wator_bm* w) {
    delete w;
    return DSR_OK;
}

// ===========================================================================
// batched form
// ===========================================================================
struct dsr_wator_batch {
    dsr_group* group;
    WatorInst* table_d;              // [max_instances] device views
    std::vector<WatorInst> table_h;  // host mirror
    bool table_pooled = false;       // the table came from the group's pool (shared arena)
    cudaStream_t capture;            // private stream used only to capture the step graph
    cudaGraphExec_t exec = nullptr;
    uint64_t exec_epoch = ~0ull;
};

static size_t table_bytes(int max_instances) { return ((size_t)max_instances * sizeof(WatorInst) + 1023) / 1024 * 1024; }

// The rest of a batch's creation once its group and table exist.
static int finish_batch(dsr_wator_batch* b, int max_instances, void* stream, dsr_wator_batch** out) {
    b->table_h.assign(max_instances, WatorInst{});
    cudaError_t e = cudaMemsetAsync(b->table_d, 0, table_bytes(max_instances), dsr__stream(stream));
    if (!e) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e) {
        dsr__set_cuda_error(e, "dsr_wator_batch_create");
        if (b->table_pooled) dsr__group_give_bytes(b->group, b->table_d, table_bytes(max_instances));
        dsr_group_destroy(b->group);
        delete b;
        return DSR_E_CUDA;
    }
    *out = b;
    return DSR_OK;
}

extern "C" int dsr_wator_batch_create(void* arena_dev, size_t arena_bytes, int max_instances, const dsr_tuning* tune,
                                      void* stream, dsr_wator_batch** out) {
    if (!arena_dev || !out || max_instances < 1 || (reinterpret_cast<uintptr_t>(arena_dev) & 255)) return DSR_E_INVALID;
    const size_t tb = table_bytes(max_instances);
    if (arena_bytes <= tb) return DSR_E_OOM;
    dsr_type_desc types[2];
    dsr_wator_types(types);
    dsr_wator_batch* b = new dsr_wator_batch;
    int rc = dsr_group_create(types, 2, static_cast<uint8_t*>(arena_dev) + tb, arena_bytes - tb, max_instances, tune,
                              stream, &b->group);
    if (rc) {
        delete b;
        return rc;
    }
    b->table_d = static_cast<WatorInst*>(arena_dev);
    return finish_batch(b, max_instances, stream, out);
}

extern "C" int dsr_wator_batch_create_shared(dsr_group* pool_of, int max_instances, const dsr_tuning* tune,
                                             void* stream, dsr_wator_batch** out) {
    if (!pool_of || !out || max_instances < 1) return DSR_E_INVALID;
    dsr_type_desc types[2];
    dsr_wator_types(types);
    dsr_wator_batch* b = new dsr_wator_batch;
    int rc = dsr_group_create_shared(types, 2, pool_of, max_instances, tune, stream, &b->group);
    if (rc) {
        delete b;
        return rc;
    }
    void* t = nullptr;
    rc = dsr__group_take_bytes(b->group, table_bytes(max_instances), &t);
    if (rc) {
        dsr_group_destroy(b->group);
        delete b;
        return rc;
    }
    b->table_d = static_cast<WatorInst*>(t);
    b->table_pooled = true;
    return finish_batch(b, max_instances, stream, out);
}

extern "C" int dsr_wator_batch_instance_bytes(const dsr_wator_batch* b, int W, int H, uint64_t n_blocks, size_t* out) {
    if (!b || !out || W < 3 || H < 3) return DSR_E_INVALID;
    return dsr_group_heap_bytes(b->group, n_blocks, ws_bytes(W, H, n_blocks * 64), out);
}

extern "C" int dsr_wator_batch_add(dsr_wator_batch* b, const dsr_wator_params* p, uint64_t n_blocks,
                                   const void* kind0_dev, void* stream, int* inst_out) {
    if (!b || !params_ok(p) || !kind0_dev || !inst_out || n_blocks == 0 || n_blocks > kMaxBlocks)
        return DSR_E_INVALID;
    int slot = -1;
    dsr_heap* heap = nullptr;
    void* extra = nullptr;
    int rc = dsr_group_add_heap(b->group, n_blocks, ws_bytes(p->W, p->H, n_blocks * 64), stream, &slot, &heap, &extra);
    if (rc) return rc;
    cudaStream_t s = dsr__stream(stream);
    if (heap->layout.n_blocks > n_blocks) {  // the intent array must cover every slot of the heap
        dsr_group_remove_heap(b->group, slot);
        return DSR_E_INVALID;
    }
    WatorInst I = carve(extra, *p, n_blocks * 64);
    rc = launch_init(heap, I, kind0_dev, s);
    if (rc) return rc;
    b->table_h[slot] = I;
    cudaError_t e = cudaMemcpyAsync(b->table_d + slot, &b->table_h[slot], sizeof(WatorInst), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_wator_batch_add");
        return DSR_E_CUDA;
    }
    *inst_out = slot;
    return DSR_OK;
}

extern "C" int dsr_wator_batch_remove(dsr_wator_batch* b, int inst) {
    if (!b || inst < 0 || inst >= (int)b->table_h.size() || !b->table_h[inst].step) return DSR_E_INVALID;
    b->table_h[inst] = WatorInst{};
    cudaError_t e = cudaMemcpy(b->table_d + inst, &b->table_h[inst], sizeof(WatorInst), cudaMemcpyHostToDevice);
    if (e) {
        dsr__set_cuda_error(e, "dsr_wator_batch_remove");
        return DSR_E_CUDA;
    }
    return dsr_group_remove_heap(b->group, inst);
}

static int issue_batch_step(dsr_wator_batch* b, cudaStream_t s) {
    dsr_group* g = b->group;
    BatchArgs a{b->table_d};
    // F2 and S2 run over the block lists of F1 and S1 (see dsr_wator_step)
    int rc = dsr__group_doall<GFishChoose>(g, FISH, a, s, true, 1);
    if (!rc) rc = dsr__group_doall<GFishMove>(g, FISH, a, s, false);
    if (!rc) rc = dsr__group_doall<GSharkStarve>(g, SHARK, a, s);
    if (!rc) rc = dsr__group_doall<GSharkChoose>(g, SHARK, a, s, true, 1);
    if (!rc) rc = dsr__group_doall<GSharkMove>(g, SHARK, a, s, false);
    return rc;
}

// One batched step is 10 launches (5 fused scans, 5 method kernels) over all
// instances; it is captured once into a CUDA graph and replayed until the set
// of instances changes.
static int ensure_graph(dsr_wator_batch* b) {
    if (b->exec_epoch == b->group->epoch) return DSR_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e) {
        dsr__set_cuda_error(e, "dsr_wator_batch_step capture");
        return DSR_E_CUDA;
    }
    const int rc = issue_batch_step(b, b->capture);
    e = cudaStreamEndCapture(b->capture, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (!e) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e) {
        dsr__set_cuda_error(e, "dsr_wator_batch_step instantiate");
        b->exec = nullptr;
        return DSR_E_CUDA;
    }
    b->exec_epoch = b->group->epoch;
    return DSR_OK;
}

extern "C" int dsr_wator_batch_prepare(dsr_wator_batch* b) {
    if (!b) return DSR_E_INVALID;
    return ensure_graph(b);
}

extern "C" int dsr_wator_batch_step(dsr_wator_batch* b, int n_steps, void* stream) {
    if (!b || n_steps < 0) return DSR_E_INVALID;
    const int rc = ensure_graph(b);
    if (rc) return rc;
    cudaStream_t s = dsr__stream(stream);
    for (int i = 0; i < n_steps; ++i) {
        cudaError_t e = cudaGraphLaunch(b->exec, s);
        if (e) {
            dsr__set_cuda_error(e, "dsr_wator_batch_step launch");
            return DSR_E_CUDA;
        }
    }
    return DSR_OK;
}

extern "C" int dsr_wator_batch_heap(dsr_wator_batch* b, int inst, dsr_heap** out) {
    if (!b || !out || inst < 0 || inst >= (int)b->table_h.size() || !b->table_h[inst].step) return DSR_E_INVALID;
    *out = b->group->heaps[inst];
    return DSR_OK;
}

extern "C" int dsr_wator_batch_kinds(dsr_wator_batch* b, int inst, void* kind_out_dev, void* stream) {
    dsr_heap* h = nullptr;
    int rc = dsr_wator_batch_heap(b, inst, &h);
    if (rc || !kind_out_dev) return rc ? rc : DSR_E_INVALID;
    return launch_kinds(h, b->table_h[inst], kind_out_dev, dsr__stream(stream));
}

extern "C" int dsr_wator_batch_group(dsr_wator_batch* b, dsr_group** out) {
    if (!b || !out) return DSR_E_INVALID;
    *out = b->group;
    return DSR_OK;
}

extern "C" int dsr_wator_batch_destroy(dsr_wator_batch* b) {
    if (!b) return DSR_E_INVALID;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    cudaStreamDestroy(b->capture);
    if (b->table_pooled) dsr__group_give_bytes(b->group, b->table_d, table_bytes((int)b->table_h.size()));
    dsr_group_destroy(b->group);
    delete b;
    return DSR_OK;
}
