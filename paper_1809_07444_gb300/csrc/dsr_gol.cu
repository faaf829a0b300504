// Game of life as an SMMO program (Fig. 6c): three do-alls per generation
// over Cell and Alive objects. Rules: B3/S23 on a torus, Moore neighbourhood.
#include "dsr_apps.h"
#include "dsr_internal.cuh"

namespace {
enum { CELL = 0, ALIVE = 1 };
enum { C_ALIVE = 0, C_COUNT = 1, C_IDX = 2 };
enum { A_X = 0, A_Y = 1 };

struct GolArgs {
    const dsr_ref* cell_ref;  // grid index -> Cell handle
    int32_t W, H;
};

// (i) do-all Cell: number of alive cells among the 8 neighbours.
struct MCount {
    typedef GolArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        const int idx = *dsr_field<int32_t>(H, CELL, self, C_IDX);
        const int x = idx % a.W, y = idx / a.W;
        int n = 0;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int ny = y + dy < 0 ? y + dy + a.H : (y + dy >= a.H ? y + dy - a.H : y + dy);
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0) continue;
                const int nx = x + dx < 0 ? x + dx + a.W : (x + dx >= a.W ? x + dx - a.W : x + dx);
                const dsr_ref c = a.cell_ref[ny * a.W + nx];
                if (c != DSR_NULL) n += *dsr_field<int32_t>(H, CELL, c, C_ALIVE);
            }
        }
        *dsr_field<int32_t>(H, CELL, self, C_COUNT) = n;
    }
};

// (ii) do-all Alive: death when the cell's count is not 2 or 3.
struct MDie {
    typedef GolArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        const int x = *dsr_field<int32_t>(H, ALIVE, self, A_X);
        const int y = *dsr_field<int32_t>(H, ALIVE, self, A_Y);
        const dsr_ref c = a.cell_ref[y * a.W + x];
        if (c == DSR_NULL) return;
        const int n = *dsr_field<int32_t>(H, CELL, c, C_COUNT);
        if (n != 2 && n != 3) {
            *dsr_field<int32_t>(H, CELL, c, C_ALIVE) = 0;
            dsr_delete(H, self);
        }
    }
};

// (iii) do-all Cell: birth of a dead cell with exactly 3 alive neighbours.
struct MBirth {
    typedef GolArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int, const Args& a, dsr_ref self) {
        int32_t* alive = dsr_field<int32_t>(H, CELL, self, C_ALIVE);
        if (*alive || *dsr_field<int32_t>(H, CELL, self, C_COUNT) != 3) return;
        *alive = 1;
        const int idx = *dsr_field<int32_t>(H, CELL, self, C_IDX);
        const dsr_ref r = dsr_new(H, ALIVE);
        if (r == DSR_NULL) return;
        *dsr_field<int32_t>(H, ALIVE, r, A_X) = idx % a.W;
        *dsr_field<int32_t>(H, ALIVE, r, A_Y) = idx / a.W;
    }
};

// One thread per cell: create the Cell and, where alive, its Alive object.
__global__ void k_gol_init(const __grid_constant__ dsr_dev_heap H, const uint8_t* alive0, dsr_ref* cell_ref,
                           int W, int Hh) {
    const int n = W * Hh;
    const int n32 = (n + 31) & ~31;  // warp-uniform trip count
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n32; i += gridDim.x * blockDim.x) {
        __syncwarp();  // whole-warp groups for dsr_new
        if (i >= n) continue;
        const int alive = alive0[i] ? 1 : 0;
        const dsr_ref c = dsr_new(H, CELL);
        cell_ref[i] = c;
        if (c != DSR_NULL) {
            *dsr_field<int32_t>(H, CELL, c, C_ALIVE) = alive;
            *dsr_field<int32_t>(H, CELL, c, C_COUNT) = 0;
            *dsr_field<int32_t>(H, CELL, c, C_IDX) = i;
        }
        if (alive) {
            const dsr_ref r = dsr_new(H, ALIVE);
            if (r != DSR_NULL) {
                *dsr_field<int32_t>(H, ALIVE, r, A_X) = i % W;
                *dsr_field<int32_t>(H, ALIVE, r, A_Y) = i / W;
            }
        }
    }
}

const int kCellFields[3] = {4, 4, 4};
const int kAliveFields[2] = {4, 4};

bool heap_matches(const dsr_heap* h) {
    const dsr_layout& L = h->layout;
    if (L.n_types < 2 || L.n_fields[CELL] != 3 || L.n_fields[ALIVE] != 2) return false;
    for (int f = 0; f < 3; ++f)
        if (L.field_bytes[CELL][f] != 4) return false;
    for (int f = 0; f < 2; ++f)
        if (L.field_bytes[ALIVE][f] != 4) return false;
    return true;
}
}  // namespace

struct dsr_gol {
    dsr_heap* heap;
    GolArgs args;
    cudaStream_t capture = nullptr;   // stream the generation is captured on
    cudaGraphExec_t exec = nullptr;   // one generation (6 launches) as a graph
};

extern "C" int dsr_gol_types(dsr_type_desc* out) {
    if (!out) return DSR_E_INVALID;
    out[0] = dsr_type_desc{"Cell", 3, kCellFields};
    out[1] = dsr_type_desc{"Alive", 2, kAliveFields};
    return DSR_OK;
}

extern "C" int dsr_gol_workspace_bytes(int W, int H, size_t* out) {
    if (!out || W < 3 || H < 3 || (int64_t)W * H > (1ll << 31)) return DSR_E_INVALID;
    *out = (size_t)W * H * sizeof(dsr_ref);
    return DSR_OK;
}

extern "C" int dsr_gol_create(dsr_heap* heap, int W, int H, const void* alive0_dev, void* workspace_dev,
                              void* stream, dsr_gol** out) {
    size_t ws;
    if (!heap || !alive0_dev || !workspace_dev || !out || dsr_gol_workspace_bytes(W, H, &ws)) return DSR_E_INVALID;
    if (!heap_matches(heap)) return DSR_E_INVALID;
    dsr_gol* g = new dsr_gol;
    g->heap = heap;
    g->args = GolArgs{static_cast<const dsr_ref*>(workspace_dev), W, H};
    const int n = W * H;
    int ctas = (n + 255) / 256;
    if (ctas > heap->sm_count * 8) ctas = heap->sm_count * 8;
    k_gol_init<<<ctas, 256, 0, dsr__stream(stream)>>>(heap->dev, static_cast<const uint8_t*>(alive0_dev),
                                                       static_cast<dsr_ref*>(workspace_dev), W, H);
    int rc = dsr__check_launch("k_gol_init");
    if (rc) {
        delete g;
        return rc;
    }
    *out = g;
    return DSR_OK;
}

static int issue_generation(dsr_gol* g, cudaStream_t s) {
    int rc = dsr__doall<MCount>(g->heap, CELL, g->args, s);
    if (!rc) rc = dsr__doall<MDie>(g->heap, ALIVE, g->args, s);
    if (!rc) rc = dsr__doall<MBirth>(g->heap, CELL, g->args, s);
    return rc;
}

// A generation's six launches take a few microseconds each on a 64 x 64
// board, so the generation is captured once into a CUDA graph (its kernel
// arguments never change) and replayed: one launch per generation.
extern "C" int dsr_gol_step(dsr_gol* g, int n_gen, void* stream) {
    if (!g || n_gen < 0) return DSR_E_INVALID;
    cudaStream_t s = dsr__stream(stream);
    if (!g->exec && n_gen > 0) {
        cudaError_t e = g->capture ? cudaSuccess : cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking);
        cudaGraph_t graph = nullptr;
        if (!e) e = cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal);
        if (e) {
            dsr__set_cuda_error(e, "dsr_gol_step capture");
            return DSR_E_CUDA;
        }
        const int rc = issue_generation(g, g->capture);
        e = cudaStreamEndCapture(g->capture, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (!e) e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e) {
            dsr__set_cuda_error(e, "dsr_gol_step instantiate");
            g->exec = nullptr;
            return DSR_E_CUDA;
        }
    }
    for (int i = 0; i < n_gen; ++i) {
        const cudaError_t e = cudaGraphLaunch(g->exec, s);
        if (e) {
            dsr__set_cuda_error(e, "dsr_gol_step launch");
            return DSR_E_CUDA;
        }
    }
    return DSR_OK;
}

extern "C" int dsr_gol_destroy(dsr_gol* g) {
    if (!g) return DSR_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->capture) cudaStreamDestroy(g->capture);
    delete g;
    return DSR_OK;
}

// dsr_parallel_do entry for the game-of-life methods. Args: dsr_gol_method_args
// = { const uint64_t* cell_ref_dev; int32_t W, H; }.
int dsr__gol_method(dsr_heap* h, int type, int method, const void* args, size_t bytes, cudaStream_t s,
                    bool with_scan) {
    if (!heap_matches(h) || !args || bytes != sizeof(GolArgs)) return DSR_E_INVALID;
    GolArgs a;
    memcpy(&a, args, sizeof a);
    switch (method) {
        case DSR_METHOD_GOL_COUNT:
            return type == CELL ? dsr__doall<MCount>(h, type, a, s, with_scan) : DSR_E_INVALID;
        case DSR_METHOD_GOL_DIE:
            return type == ALIVE ? dsr__doall<MDie>(h, type, a, s, with_scan) : DSR_E_INVALID;
        case DSR_METHOD_GOL_BIRTH:
            return type == CELL ? dsr__doall<MBirth>(h, type, a, s, with_scan) : DSR_E_INVALID;
        default:
            return DSR_E_INVALID;
    }
}

// ===========================================================================
// batched form: many game-of-life instances in one heap group
// ===========================================================================
#include "dsr_group.cuh"

namespace {
struct GolBatchArgs {
    const GolArgs* table;  // slot -> instance view (cell_ref == nullptr: unused slot)
};
struct GCount {
    typedef GolBatchArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int T, const Args& a, dsr_ref s, uint32_t h) {
        MCount::run(H, T, a.table[h], s);
    }
};
struct GDie {
    typedef GolBatchArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int T, const Args& a, dsr_ref s, uint32_t h) {
        MDie::run(H, T, a.table[h], s);
    }
};
struct GBirth {
    typedef GolBatchArgs Args;
    static __device__ void run(const dsr_dev_heap& H, int T, const Args& a, dsr_ref s, uint32_t h) {
        MBirth::run(H, T, a.table[h], s);
    }
};
size_t gol_table_bytes(int n) { return ((size_t)n * sizeof(GolArgs) + 1023) / 1024 * 1024; }
}  // namespace

struct dsr_gol_batch {
    dsr_group* group;
    GolArgs* table_d;
    std::vector<GolArgs> table_h;
    bool table_pooled = false;  // the table came from the group's pool (shared arena)
    cudaStream_t capture;
    cudaGraphExec_t exec = nullptr;
    uint64_t exec_epoch = ~0ull;
};

// The rest of a batch's creation once its group and table exist.
static int finish_gol_batch(dsr_gol_batch* b, int max_instances, void* stream, dsr_gol_batch** out) {
    b->table_h.assign(max_instances, GolArgs{nullptr, 0, 0});
    cudaError_t e = cudaMemsetAsync(b->table_d, 0, gol_table_bytes(max_instances), dsr__stream(stream));
    if (!e) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e) {
        dsr__set_cuda_error(e, "dsr_gol_batch_create");
        if (b->table_pooled) dsr__group_give_bytes(b->group, b->table_d, gol_table_bytes(max_instances));
        dsr_group_destroy(b->group);
        delete b;
        return DSR_E_CUDA;
    }
    *out = b;
    return DSR_OK;
}

extern "C" int dsr_gol_batch_create(void* arena_dev, size_t arena_bytes, int max_instances, const dsr_tuning* tune,
                                    void* stream, dsr_gol_batch** out) {
    if (!arena_dev || !out || max_instances < 1 || (reinterpret_cast<uintptr_t>(arena_dev) & 255)) return DSR_E_INVALID;
    const size_t tb = gol_table_bytes(max_instances);
    if (arena_bytes <= tb) return DSR_E_OOM;
    dsr_type_desc types[2];
    dsr_gol_types(types);
    dsr_gol_batch* b = new dsr_gol_batch;
    int rc = dsr_group_create(types, 2, static_cast<uint8_t*>(arena_dev) + tb, arena_bytes - tb, max_instances, tune,
                              stream, &b->group);
    if (rc) {
        delete b;
        return rc;
    }
    b->table_d = static_cast<GolArgs*>(arena_dev);
    return finish_gol_batch(b, max_instances, stream, out);
}

extern "C" int dsr_gol_batch_create_shared(dsr_group* pool_of, int max_instances, const dsr_tuning* tune,
                                           void* stream, dsr_gol_batch** out) {
    if (!pool_of || !out || max_instances < 1) return DSR_E_INVALID;
    dsr_type_desc types[2];
    dsr_gol_types(types);
    dsr_gol_batch* b = new dsr_gol_batch;
    int rc = dsr_group_create_shared(types, 2, pool_of, max_instances, tune, stream, &b->group);
    if (rc) {
        delete b;
        return rc;
    }
    void* t = nullptr;
    rc = dsr__group_take_bytes(b->group, gol_table_bytes(max_instances), &t);
    if (rc) {
        dsr_group_destroy(b->group);
        delete b;
        return rc;
    }
    b->table_d = static_cast<GolArgs*>(t);
    b->table_pooled = true;
    return finish_gol_batch(b, max_instances, stream, out);
}

extern "C" int dsr_gol_batch_instance_bytes(const dsr_gol_batch* b, int W, int H, uint64_t n_blocks, size_t* out) {
    size_t ws;
    if (!b || !out || dsr_gol_workspace_bytes(W, H, &ws)) return DSR_E_INVALID;
    return dsr_group_heap_bytes(b->group, n_blocks, ws, out);
}

extern "C" int dsr_gol_batch_add(dsr_gol_batch* b, int W, int H, uint64_t n_blocks, const void* alive0_dev,
                                 void* stream, int* inst_out) {
    size_t ws;
    if (!b || !alive0_dev || !inst_out || n_blocks == 0 || dsr_gol_workspace_bytes(W, H, &ws)) return DSR_E_INVALID;
    int slot = -1;
    dsr_heap* heap = nullptr;
    void* extra = nullptr;
    int rc = dsr_group_add_heap(b->group, n_blocks, ws, stream, &slot, &heap, &extra);
    if (rc) return rc;
    cudaStream_t s = dsr__stream(stream);
    const int n = W * H;
    int ctas = (n + 255) / 256;
    if (ctas > heap->sm_count * 8) ctas = heap->sm_count * 8;
    k_gol_init<<<ctas, 256, 0, s>>>(heap->dev, static_cast<const uint8_t*>(alive0_dev), static_cast<dsr_ref*>(extra),
                                    W, H);
    rc = dsr__check_launch("k_gol_init");
    if (rc) return rc;
    b->table_h[slot] = GolArgs{static_cast<const dsr_ref*>(extra), W, H};
    cudaError_t e = cudaMemcpyAsync(b->table_d + slot, &b->table_h[slot], sizeof(GolArgs), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) {
        dsr__set_cuda_error(e, "dsr_gol_batch_add");
        return DSR_E_CUDA;
    }
    *inst_out = slot;
    return DSR_OK;
}

extern "C" int dsr_gol_batch_remove(dsr_gol_batch* b, int inst) {
    if (!b || inst < 0 || inst >= (int)b->table_h.size() || !b->table_h[inst].cell_ref) return DSR_E_INVALID;
    b->table_h[inst] = GolArgs{nullptr, 0, 0};
    cudaError_t e = cudaMemcpy(b->table_d + inst, &b->table_h[inst], sizeof(GolArgs), cudaMemcpyHostToDevice);
    if (e) {
        dsr__set_cuda_error(e, "dsr_gol_batch_remove");
        return DSR_E_CUDA;
    }
    return dsr_group_remove_heap(b->group, inst);
}

// One batched generation: three group do-alls (6 launches), captured into a
// CUDA graph once per set of instances.
static int ensure_gol_graph(dsr_gol_batch* b) {
    if (b->exec_epoch == b->group->epoch) return DSR_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e) {
        dsr__set_cuda_error(e, "dsr_gol_batch_step capture");
        return DSR_E_CUDA;
    }
    GolBatchArgs a{b->table_d};
    int rc = dsr__group_doall<GCount>(b->group, CELL, a, b->capture);
    if (!rc) rc = dsr__group_doall<GDie>(b->group, ALIVE, a, b->capture);
    if (!rc) rc = dsr__group_doall<GBirth>(b->group, CELL, a, b->capture);
    e = cudaStreamEndCapture(b->capture, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (!e) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e) {
        dsr__set_cuda_error(e, "dsr_gol_batch_step instantiate");
        b->exec = nullptr;
        return DSR_E_CUDA;
    }
    b->exec_epoch = b->group->epoch;
    return DSR_OK;
}

extern "C" int dsr_gol_batch_prepare(dsr_gol_batch* b) {
    if (!b) return DSR_E_INVALID;
    return ensure_gol_graph(b);
}

extern "C" int dsr_gol_batch_step(dsr_gol_batch* b, int n_gen, void* stream) {
    if (!b || n_gen < 0) return DSR_E_INVALID;
    const int rc = ensure_gol_graph(b);
    if (rc) return rc;
    cudaStream_t s = dsr__stream(stream);
    for (int i = 0; i < n_gen; ++i) {
        cudaError_t e = cudaGraphLaunch(b->exec, s);
        if (e) {
            dsr__set_cuda_error(e, "dsr_gol_batch_step launch");
            return DSR_E_CUDA;
        }
    }
    return DSR_OK;
}

extern "C" int dsr_gol_batch_heap(dsr_gol_batch* b, int inst, dsr_heap** out) {
    if (!b || !out || inst < 0 || inst >= (int)b->table_h.size() || !b->table_h[inst].cell_ref) return DSR_E_INVALID;
    *out = b->group->heaps[inst];
    return DSR_OK;
}

extern "C" int dsr_gol_batch_group(dsr_gol_batch* b, dsr_group** out) {
    if (!b || !out) return DSR_E_INVALID;
    *out = b->group;
    return DSR_OK;
}

extern "C" int dsr_gol_batch_destroy(dsr_gol_batch* b) {
    if (!b) return DSR_E_INVALID;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    cudaStreamDestroy(b->capture);
    if (b->table_pooled) dsr__group_give_bytes(b->group, b->table_d, gol_table_bytes((int)b->table_h.size()));
    dsr_group_destroy(b->group);
    delete b;
    return DSR_OK;
}
