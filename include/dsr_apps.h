/*
 * dsr_apps.h -- C ABI of the SMMO applications that drive the heap.
 *
 * The paper evaluates its allocator with SMMO applications (Fig. 6): among
 * them game-of-life (cellular automaton), wator (agent-based predator-prey),
 * nbody / collisions (particle systems), traffic (Nagel-Schreckenberg) and
 * sugarscape (Epstein-Axtell). It names them without rules;
 * the rules implemented here are stated at each entry point and are the same
 * as the oracle's.
 *
 * Each application keeps its objects in a dsr_heap created with the type
 * descriptors returned by its *_types call (type ids in that order), plus a
 * caller-owned device workspace of *_workspace_bytes bytes (256-byte
 * aligned). Steps are queued on `stream`; each step is a fixed sequence of
 * parallel do-alls (dsr_parallel_do with the method ids below). Conventions
 * for pointers, ownership and status codes are those of dsr.h.
 */
#ifndef DSR_APPS_H
#define DSR_APPS_H

#include "dsr.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- game of life --------------------------------------------------------
 * Conway's B3/S23 on a W x H torus, Moore neighbourhood. Types: 0 Cell
 * {alive, count, idx} with idx = y*W + x, 1 Alive {x, y}. One generation is
 * three do-alls:
 *   DSR_METHOD_GOL_COUNT (Cell):  count = alive neighbours
 *   DSR_METHOD_GOL_DIE   (Alive): if its cell's count is not 2 or 3 the cell
 *                                 dies and the Alive object deletes itself
 *   DSR_METHOD_GOL_BIRTH (Cell):  a dead cell with count 3 becomes alive and
 *                                 creates an Alive object.
 * Workspace: uint64 Cell handle per cell. */
enum { DSR_METHOD_GOL_COUNT = 100, DSR_METHOD_GOL_DIE = 101, DSR_METHOD_GOL_BIRTH = 102 };
typedef struct dsr_gol dsr_gol;
int dsr_gol_types(dsr_type_desc* out /* 2 entries */);
int dsr_gol_workspace_bytes(int W, int H, size_t* out);
/* alive0_dev: device uint8[W*H], 1 = alive. Allocates the Cells and the
 * initial Alive objects inside the heap. */
int dsr_gol_create(dsr_heap* heap, int W, int H, const void* alive0_dev, void* workspace_dev, void* stream,
                   dsr_gol** out);
/* The first call captures one generation (its six launches) into a CUDA
 * graph on a stream of its own; every generation is then one graph launch
 * on `stream`. Make the first call outside any stream capture. */
int dsr_gol_step(dsr_gol* g, int n_gen, void* stream);
int dsr_gol_destroy(dsr_gol* g);

/* Batched game of life: many instances, each with its own heap in one heap
 * group, advanced together by three group do-alls per generation captured
 * into a CUDA graph (same conventions as the batched wa-tor below). */
typedef struct dsr_gol_batch dsr_gol_batch;
int dsr_gol_batch_create(void* arena_dev, size_t arena_bytes, int max_instances, const dsr_tuning* tune, void* stream,
                         dsr_gol_batch** out);
int dsr_gol_batch_instance_bytes(const dsr_gol_batch* b, int W, int H, uint64_t n_blocks, size_t* out);
int dsr_gol_batch_add(dsr_gol_batch* b, int W, int H, uint64_t n_blocks, const void* alive0_dev, void* stream,
                      int* inst_out);
int dsr_gol_batch_remove(dsr_gol_batch* b, int inst);
/* A batch in the arena of an existing group (dsr_group_create_shared): its
 * instances compete for the same free bytes as that group's heaps, e.g. a
 * wa-tor batch's (dsr_wator_batch_group). */
int dsr_gol_batch_create_shared(dsr_group* pool_of, int max_instances, const dsr_tuning* tune, void* stream,
                                dsr_gol_batch** out);
/* Capture the batched generation into its CUDA graph now if the set of
 * instances changed since the last capture (dsr_gol_batch_step does it
 * otherwise, on its first call after the change). Host work only. */
int dsr_gol_batch_prepare(dsr_gol_batch* b);
int dsr_gol_batch_step(dsr_gol_batch* b, int n_gen, void* stream);
int dsr_gol_batch_heap(dsr_gol_batch* b, int inst, dsr_heap** out);
int dsr_gol_batch_group(dsr_gol_batch* b, dsr_group** out);
int dsr_gol_batch_destroy(dsr_gol_batch* b);

/* ---- wa-tor ----------------------------------------------------------------
 * W x H torus, von Neumann neighbours in the order N (y-1), E (x+1), S (y+1),
 * W (x-1); cell index c = y*W + x. Types: 0 Fish {x, y, timer}, 1 Shark
 * {x, y, timer, energy}. Random choices: r = SplitMix64 counter draw keyed on
 * (seed, stream 0 for fish / 1 for sharks, step, mover's cell); a mover picks
 * candidate (r mod k) of its k candidates. One step is five do-alls:
 *   F1 (Fish):  timer += 1; candidates = empty neighbours; claim the pick
 *               (the lowest mover cell index wins a contested cell)
 *   F2 (Fish):  winners move; timer >= fish_breed: leave a new Fish
 *               (timer 0) behind and reset timer
 *   S0 (Shark): energy -= 1; at 0 the shark is deleted
 *   S1 (Shark): timer += 1; candidates = neighbouring fish, else empty
 *               neighbours; claim as F1
 *   S2 (Shark): winners move; a fish in the target is deleted and energy +=
 *               shark_gain; timer >= shark_breed: leave a new Shark (timer 0,
 *               energy shark_energy0) behind and reset timer.
 * Workspace (dsr_wator_workspace_bytes, which depends on the heap): a uint32
 * grid word per cell (0 empty, else (handle << 2) | kind; heaps of at most
 * 2^24 blocks), a uint32 claim word per cell (the lowest mover cell that
 * claimed it; the winner resets it when it moves), the step counter, and a
 * uint32 intent per object slot of the heap (the target an agent chose in
 * F1 / S1, read back in F2 / S2 with the agent's fields).
 * Each successful move (F2 and S2 winners) adds one to the heap's
 * DSR_CTR_APP0 event counter. */
enum {
    DSR_METHOD_WATOR_F1 = 200,
    DSR_METHOD_WATOR_F2 = 201,
    DSR_METHOD_WATOR_S0 = 202,
    DSR_METHOD_WATOR_S1 = 203,
    DSR_METHOD_WATOR_S2 = 204
};
typedef struct {
    int32_t W, H;
    uint64_t seed;
    int32_t fish_breed;     /* 3 */
    int32_t shark_breed;    /* 10 */
    int32_t shark_energy0;  /* 5 */
    int32_t shark_gain;     /* 3 */
} dsr_wator_params;
typedef struct dsr_wator dsr_wator;
int dsr_wator_types(dsr_type_desc* out /* 2 entries */);
/* Workspace bytes for a W x H torus whose agents live in `heap`. */
int dsr_wator_workspace_bytes(const dsr_heap* heap, int W, int H, size_t* out);
/* kind0_dev: device uint8[W*H]: 0 empty, 1 fish, 2 shark. Initial fish have
 * timer 0; sharks timer 0 and energy shark_energy0. */
int dsr_wator_create(dsr_heap* heap, const dsr_wator_params* p, const void* kind0_dev, void* workspace_dev,
                     void* stream, dsr_wator** out);
/* Advances n_steps steps on `stream` (each step: F1, F2, S0, S1, S2 as
 * do-alls). A step is replayed from a CUDA graph of its 8 launches that the
 * handle captures on first use on a private stream (one for untimed steps,
 * one for the current dsr_wator_phase_timing / _phase_select setting, which
 * is captured when that setting is made); while `stream` is itself being
 * captured, the kernels are launched into that capture instead. If a
 * capture fails the handle launches kernel by kernel from then on. */
int dsr_wator_step(dsr_wator* w, int n_steps, void* stream);
/* A handle over a heap and workspace that already hold a wa-tor state, with
 * no initialisation: resuming from a checkpoint. A checkpoint of a wa-tor
 * run is the bytes of its heap arena and of its workspace (no pointer is
 * stored inside either; handles are block and slot numbers, the random draws
 * are keyed on the step counter in the workspace). Restore by creating a
 * heap of the same types, size and tuning over a new arena (the same layout
 * follows), copying the saved arena bytes over it after the creation's reset
 * has run, copying the workspace bytes, and attaching. No counterpart in the
 * paper. */
int dsr_wator_attach(dsr_heap* heap, const dsr_wator_params* p, void* workspace_dev, dsr_wator** out);
/* Device uint8[W*H] occupancy snapshot (0/1/2) of the current state. */
int dsr_wator_kinds(dsr_wator* w, void* kind_out_dev, void* stream);
int dsr_wator_destroy(dsr_wator* w);
/* Per-phase timing (a measurement aid; the paper times whole runs). With
 * max_steps > 0, creates 11 CUDA events per step for the next max_steps
 * steps (device current = the heap's); each of those steps then records them
 * on its stream at its start and after every scan and method kernel. 0 frees
 * them. Each recorded event also lengthens the step on the device: on a
 * GB300, the 11 events of a 2048 x 2048 step added 5-20 us to its 0.29 ms
 * (dsr_wator_phase_select records two). DSR_E_CUDA if an event cannot be
 * created (none are kept). */
int dsr_wator_phase_timing(dsr_wator* w, int max_steps);
/* Restricts the events of dsr_wator_phase_timing to the method kernel of one
 * phase: phase 0..4 (F1, F2, S0, S1, S2) records only the two events around
 * that kernel, -1 (the default) records all 11. Starts a new window (steps
 * recorded before are dropped); dsr_wator_phase_times then reports that
 * phase's method time and 0 for the other entries. DSR_E_INVALID for another
 * phase value. */
int dsr_wator_phase_select(dsr_wator* w, int phase);
/* Waits for the last recorded step, then writes the summed device
 * milliseconds of the steps recorded since the last call: out_ms[0..4] the
 * method kernels of F1, F2, S0, S1, S2, out_ms[5..9] their scans (the times
 * between a phase's start and its method kernel); *steps = the number of
 * steps. Starts a new window (the events are reused). */
int dsr_wator_phase_times(dsr_wator* w, double* out_ms /* 10 */, int* steps);

/* Wa-tor on the BitmapAlloc comparator (dsr_bm_heap_* in dsr.h): the same
 * rules and workspace as dsr_wator_*, with Fish and Shark objects in the
 * comparator's per-type arrays (types 0 and 1 as dsr_wator_types gives). */
typedef struct dsr_wator_bm dsr_wator_bm;
int dsr_wator_bm_workspace_bytes(const dsr_bm_heap* heap, int W, int H, size_t* out);
int dsr_wator_bm_create(dsr_bm_heap* heap, const dsr_wator_params* p, const void* kind0_dev, void* workspace_dev,
                        void* stream, dsr_wator_bm** out);
int dsr_wator_bm_step(dsr_wator_bm* w, int n_steps, void* stream);
int dsr_wator_bm_destroy(dsr_wator_bm* w);

/* ---- wa-tor without dynamic allocation ------------------------------------
 * The "Baseline AOS/SOA" comparators of Section 4: the agents live in
 * per-cell arrays (aos = 0: one array per field; aos = 1: one 12-byte struct
 * per cell), each phase is a kernel over all cells, and a move copies the
 * agent's data to the target cell. Same rules, random draws and claim keys
 * as dsr_wator_*, hence the same state after every step. The workspace
 * (device, 256-byte aligned, dsr_wator_static_bytes) holds the cells, the
 * claim and intent arrays and a visit counter. The step number is kept on
 * the host. */
typedef struct dsr_wator_static dsr_wator_static;
int dsr_wator_static_bytes(int W, int H, int aos, size_t* out);
int dsr_wator_static_create(const dsr_wator_params* p, const void* kind0_dev, void* workspace_dev, int aos,
                            void* stream, dsr_wator_static** out);
int dsr_wator_static_step(dsr_wator_static* w, int n_steps, void* stream);
/* Adds the object-state hash of dsr_heap_hash (Fish {x, y, timer}, Shark
 * {x, y, timer, energy}) to hash_dev[0] (fish) and hash_dev[1] (sharks). */
int dsr_wator_static_hash(dsr_wator_static* w, void* hash_dev, void* stream);
/* Per-cell state: kind uint8 (0 empty, 1 fish, 2 shark), timer and energy
 * int32 (0 where unused), each W*H entries in cell order. */
int dsr_wator_static_state(dsr_wator_static* w, void* kind_dev, void* timer_dev, void* energy_dev, void* stream);
/* Agents visited by the phase kernels so far (synchronises the device). */
int dsr_wator_static_visits(dsr_wator_static* w, uint64_t* out);
int dsr_wator_static_destroy(dsr_wator_static* w);

/* ---- batched wa-tor ----------------------------------------------------------
 * Many independent wa-tor instances (each with its own sizes, parameters and
 * seed) advance together: every instance has its own heap in a heap group
 * (dsr_group_* in dsr.h) carved from one caller-owned arena, and one batched
 * step is five group do-alls (one fused scan and one method kernel each) over
 * all instances, captured once into a CUDA graph and replayed until an
 * instance is added or removed. Each instance follows exactly the rules and
 * results of the plain form. The arena must be 256-byte aligned; its first
 * bytes hold the instance table. */
typedef struct dsr_wator_batch dsr_wator_batch;
int dsr_wator_batch_create(void* arena_dev, size_t arena_bytes, int max_instances, const dsr_tuning* tune,
                           void* stream, dsr_wator_batch** out);
/* Arena bytes an instance of W x H with a heap of n_blocks blocks takes. */
int dsr_wator_batch_instance_bytes(const dsr_wator_batch* b, int W, int H, uint64_t n_blocks, size_t* out);
/* Add an instance (kind0_dev as for dsr_wator_create) whose heap has at least
 * n_blocks blocks; *inst_out receives its slot. DSR_E_OOM when the arena has
 * no free range large enough or all slots are taken. Synchronises `stream`. */
int dsr_wator_batch_add(dsr_wator_batch* b, const dsr_wator_params* p, uint64_t n_blocks, const void* kind0_dev,
                        void* stream, int* inst_out);
/* Remove an instance and return its bytes. The caller must have finished all
 * work on it (synchronise the stream first). */
int dsr_wator_batch_remove(dsr_wator_batch* b, int inst);
/* n_steps batched steps of every instance, queued on `stream`. */
/* A batch in the arena of an existing group (dsr_group_create_shared), e.g. a
 * game-of-life batch's (dsr_gol_batch_group). */
int dsr_wator_batch_create_shared(dsr_group* pool_of, int max_instances, const dsr_tuning* tune, void* stream,
                                  dsr_wator_batch** out);
/* Capture the batched step into its CUDA graph now if the set of instances
 * changed since the last capture (otherwise dsr_wator_batch_step does it).
 * Host work only. */
int dsr_wator_batch_prepare(dsr_wator_batch* b);
int dsr_wator_batch_step(dsr_wator_batch* b, int n_steps, void* stream);
/* The heap of an instance (for dsr_heap_hash, dsr_heap_dump, dsr_heap_stats). */
int dsr_wator_batch_heap(dsr_wator_batch* b, int inst, dsr_heap** out);
int dsr_wator_batch_kinds(dsr_wator_batch* b, int inst, void* kind_out_dev, void* stream);
int dsr_wator_batch_group(dsr_wator_batch* b, dsr_group** out);
int dsr_wator_batch_destroy(dsr_wator_batch* b);

/* ---- n-body with merging collisions ------------------------------------
 * Fig. 6b ("collisions") and 6d ("nbody"); Fig. 1 names an Euler time step.
 * Types: 0 Body {id (int32); x, y, z, vx, vy, vz, m (float); then the low
 * words xl, yl, zl, vxl, vyl, vzl, ml (float)}: each state component is the
 * FP32 pair (high word, low word) whose sum is its value, about 48
 * significant bits. One step:
 *   a_i = G sum_j m_j d_ij / (|d_ij|^2 + eps^2)^(3/2); v += a dt; x += v dt;
 * then, on the new positions, the partner of i is the body with the lowest
 * id j != i closer than r_merge; mutual partners merge (the lower id keeps
 * the summed mass and the mass-weighted mean position and velocity, the
 * higher id is deleted).
 * Arithmetic: the update, the merge distance test (FP32 candidates, FP64
 * decision) and the merges run in FP64. The all-pairs sum runs in
 *   DSR_NBODY_PAIRS_FP32  FP32 on the high words, except for pairs closer
 *                         than r_near (an FP32 test on the high words), which
 *                         are summed in FP64 from the full state in the order
 *                         of the partners' ids; r_near = 0 leaves every pair
 *                         in FP32;
 *   DSR_NBODY_PAIRS_FP64  FP64 from the full state for every pair (r_near is
 *                         not used).
 * Close encounters amplify rounding: on the 65,536-body workload the FP32
 * pair mode stays within 1e-4 relative of an FP64 reference for 23 steps,
 * the FP64 pair mode for all 50.
 * Each step sorts the live bodies by cell of a K^3 grid over the unit cube
 * (cells at least as wide as r_near and r_merge, K <= 32; positions outside
 * the cube fall in the border cells), so that tiles of the all-pairs sum are
 * spatially compact: tiles far from a row skip the near test, and the near
 * field and the merge-partner search look only at the 27 cells around a
 * body. Every sum has a fixed order: a step is deterministic.
 * Workspace (dsr_nbody_workspace_bytes): the cell counts and offsets, the
 * sorted per-body arrays for all M * 64 slots of the heap (rounded up to
 * 1024), the slice buffers of the split all-pairs kernels (sized from the
 * device's SM count and the kernels' occupancy, so query it on the device
 * that will run the step), and a merge log of log_cap entries. */
#define DSR_NBODY_PAIRS_FP32 0
#define DSR_NBODY_PAIRS_FP64 1
typedef struct {
    double G, eps, dt, r_merge, r_near;
    int32_t pair_precision; /* DSR_NBODY_PAIRS_FP32 or DSR_NBODY_PAIRS_FP64 */
    int32_t pad_;
} dsr_nbody_params;
typedef struct dsr_nbody dsr_nbody;
int dsr_nbody_types(dsr_type_desc* out /* 1 entry */);
int dsr_nbody_workspace_bytes(const dsr_heap* heap, uint64_t log_cap, size_t* out);
/* rows_dev: device float[n_bodies][7] = (x, y, z, vx, vy, vz, m); body i gets id i. */
int dsr_nbody_create(dsr_heap* heap, const dsr_nbody_params* p, const void* rows_dev, int n_bodies,
                     void* workspace_dev, uint64_t log_cap, void* stream, dsr_nbody** out);
int dsr_nbody_step(dsr_nbody* nb, int n_steps, void* stream);
/* Device pointers to the merge log (int32[log_cap][3]: step, survivor id,
 * absorbed id, in arbitrary order within a step) and its uint64 count. */
int dsr_nbody_merge_log(dsr_nbody* nb, void** log_dev, void** count_dev);
/* Device pointer to the uint32 count of near-field pairs (closer than r_near,
 * each counted from both bodies) of the last step. */
int dsr_nbody_near_pairs(dsr_nbody* nb, void** count_dev);
int dsr_nbody_destroy(dsr_nbody* nb);

/* Allocation-free n-body step (the paper has no counterpart). Same steps and
 * results as dsr_nbody_step, for callers that cannot call cudaMalloc: code
 * that runs where device allocation is not allowed or not available, such as
 * a plugin that is handed its device memory by a host program that owns all
 * of it and forbids allocations of its own. Instead of a
 * caller-allocated workspace, the scratch of a step (cell counts and
 * offsets, 384 KB; the sorted state before and after the update, handles,
 * partners and far-field sums, 188 bytes per slot) and the step counter live
 * in a static device array inside this library, sized for
 * DSR_NOALLOC_MAX_SLOTS slots (about 3.5 MB), which every GPU that loads the
 * library holds until the process exits. The call allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.
 *   heap        a heap whose type 0 is Body (dsr_nbody_types) and whose block
 *               count times 64 is at most DSR_NOALLOC_MAX_SLOTS; a larger
 *               heap is rejected with DSR_E_TOO_LARGE.
 *   step0       the step number recorded in the merge log for the first of
 *               the n_steps steps.
 *   log_dev     device int32[log_cap][3] merge log (may be NULL if log_cap
 *               is 0); log_count_dev: device uint64 that receives, added to
 *               its current value, the number of merges.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and later calls reuse it;
 * make that first call before any stream capture. The address belongs to
 * the device's current context: after cudaDeviceReset (or any teardown of
 * the primary context) it is stale, so do not call this entry point again
 * in that process. Every call shares the one array and it keeps the last
 * call's contents (the step counter is set at the start of each call): calls
 * that overlap on the GPU (other streams, or other threads) race, so order
 * them on one stream. */
#define DSR_NOALLOC_MAX_SLOTS 16384
int dsr_nbody_step_noalloc(dsr_heap* heap, const dsr_nbody_params* p, int n_steps, uint64_t step0, void* log_dev,
                           uint64_t log_cap, void* log_count_dev, void* stream);

/* ---- traffic (Fig. 6g: the Nagel-Schreckenberg model) --------------------
 * R single-lane roads of L cells, parallel update, integer state. Types:
 * 0 Car {road, x, v}, 1 Source {road, entered, blocked} (one per open road).
 * Step t (from 0), with occupancy read as it was at the start of the step:
 *   do-all Car:    v1 = min(v + 1, vmax); g = free cells ahead of the car
 *                  up to v1 cells (open road: cells past the end are free;
 *                  periodic road: the road wraps); v2 = min(v1, g);
 *                  v3 = max(v2 - 1, 0) if the draw rand(seed, 5, t,
 *                  road * L + x) is below p, else v2; x' = x + v3; on an
 *                  open road a car with x' >= L leaves (is deleted), on a
 *                  periodic road x' wraps.
 *   do-all Source: (open roads) if cell 0 is free after the cars moved and
 *                  the draw rand(seed, 6, t, road) is below alpha, a new
 *                  Car(road, 0, v_entry) enters and `entered` grows by 1; if
 *                  a car holds cell 0, `blocked` grows by 1.
 * rand is the counter-based draw of the wa-tor rules (SplitMix64 outputs
 * keyed by seed, stream, step and cell); "below p" means (r >> 32) < p_thr
 * with p_thr = floor(p * 2^32) (2^32 for p = 1). Event counters
 * (dsr_heap_counters): APP0 cars entered, APP1 cars that left, APP2 cars
 * that moved, APP3 the sum of the new velocities (flow x R x L per step).
 * Workspace: two byte grids of R * L cells (each rounded up to 256 bytes).
 * Requires 1 <= vmax <= 127, L > vmax, 0 <= v_entry <= vmax. */
typedef struct {
    int32_t R, L, vmax, v_entry, periodic, pad_;
    uint64_t seed, p_thr, a_thr;
} dsr_traffic_params;
typedef struct dsr_traffic dsr_traffic;
int dsr_traffic_types(dsr_type_desc* out /* 2 entries */);
int dsr_traffic_workspace_bytes(const dsr_traffic_params* p, size_t* out);
/* v0_dev: device int8[R * L], -1 for an empty cell, else the initial
 * velocity of the car there (capped at vmax). */
int dsr_traffic_create(dsr_heap* heap, const dsr_traffic_params* p, const void* v0_dev, void* workspace_dev,
                       void* stream, dsr_traffic** out);
int dsr_traffic_step(dsr_traffic* t, int n_steps, void* stream);
/* Device pointer to the current occupancy grid (uint8[R * L], 1 = car). */
int dsr_traffic_occupancy(const dsr_traffic* t, const void** grid_dev);
int dsr_traffic_destroy(dsr_traffic* t);

/* ---- sugarscape (Fig. 6f; Epstein and Axtell's rules M, G_alpha, R) -----
 * W x H torus of sugar cells (capacity 0..4, sugar starts at capacity and
 * grows back by alpha a step up to it). Type: 0 Agent {x, y, sugar,
 * metabolism, vision, age, max_age, dead}. Step t:
 *   A1 do-all Agent: target = among the own cell and the cells up to
 *      `vision` away in the order N (y-1), E (x+1), S (y+1), W (x-1) that no
 *      agent occupies, the most sugar, then the nearest, then candidate
 *      (r >> 32) mod k with r = rand(seed, 12, t, own cell); a target other
 *      than the own cell is claimed, the lowest own cell index wins.
 *   A2 do-all Agent: the winner moves; every agent takes all the sugar of its
 *      cell, pays its metabolism and ages by 1; it dies (dead = 1) if its
 *      sugar is below 0 or its age reached max_age.
 *   A3 do-all Agent: a dead agent draws c = (rand(seed, 13, t, own) >> 32)
 *      mod (W * H) and claims c if no agent occupies it (lowest own wins).
 *   A4 do-all Agent: a dead agent is replaced by a new agent (age 0; sugar,
 *      metabolism, vision, max_age = lo + (r >> 32) mod (hi - lo + 1) with
 *      r = rand(seed, 8..11, t, new cell)) at c if it won c, else in its
 *      own cell, and deletes itself.
 * rand as for the wa-tor rules. Workspace (dsr_sugarscape_workspace_bytes,
 * which depends on the heap): per-cell capacity, occupancy, last-harvest
 * step and two claim words, a target per heap slot, and event counters.
 * Requires W, H >= 2 * vision_hi + 1, vision_hi <= 64, W * H < 2^31; at
 * most 2^28 - 2 steps (DSR_E_INVALID beyond). */
typedef struct {
    int32_t W, H;
    uint64_t seed;
    int32_t alpha;
    int32_t endow_lo, endow_hi, metab_lo, metab_hi, vision_lo, vision_hi, age_lo, age_hi;
} dsr_sugarscape_params;
typedef struct dsr_sugarscape dsr_sugarscape;
int dsr_sugarscape_types(dsr_type_desc* out /* 1 entry */);
int dsr_sugarscape_workspace_bytes(const dsr_heap* heap, const dsr_sugarscape_params* p, size_t* out);
/* cap_dev: device uint8[W * H]; agents0_dev: device int32[n_agents][7] =
 * (x, y, sugar, metabolism, vision, age, max_age) at distinct cells. Both
 * are read by kernels queued on `stream`: keep them until those have run. */
int dsr_sugarscape_create(dsr_heap* heap, const dsr_sugarscape_params* p, const void* cap_dev,
                          const void* agents0_dev, int64_t n_agents, void* workspace_dev, void* stream,
                          dsr_sugarscape** out);
int dsr_sugarscape_step(dsr_sugarscape* s, int n_steps, void* stream);
/* Cumulative events (host uint64[5]): moves, agents starved, agents that
 * reached their maximum age, replacements placed away from the dead agent's
 * cell, sugar harvested. Synchronises `stream`. */
int dsr_sugarscape_events(dsr_sugarscape* s, void* stream, uint64_t* out);
/* The sugar of every cell at the start of the next step (device int32[W*H]). */
int dsr_sugarscape_sugar(dsr_sugarscape* s, void* out_dev, void* stream);
int dsr_sugarscape_destroy(dsr_sugarscape* s);

#ifdef __cplusplus
}
#endif
#endif /* DSR_APPS_H */
