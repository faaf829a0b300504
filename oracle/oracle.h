/*
 * Oracle for the DynaSOAr hot path (Springer, "DynaSOAr: Accelerating
 * Single-Method Multiple-Objects Applications on GPUs").
 *
 * TEST INFRASTRUCTURE ONLY. Plain, slow C++ that states what the GPU path
 * must compute. Single-threaded, except that the n-body force and partner
 * loops may hand whole rows to std::thread workers (orc_set_threads): each
 * row is still summed by one thread in index order, so the result does not
 * depend on the thread count. Only the test suite, the smoke check and the
 * bench's CPU-baseline leg may load it. It shares no code, header, table or
 * constant generator with the CUDA library; it implements its own copy of the
 * counter-based generator from the published SplitMix64 definition.
 *
 * Contents
 *   - SplitMix64 counter generator (Steele, Lea & Flood, OOPSLA 2014).
 *   - Order-independent object-state hash.
 *   - Hierarchical bitmap, sequential model with a container-width parameter
 *     (Section 3, "Data Structure", container-consistency equation, Alg. 2,
 *     Fig. 5 uses width 4).
 *   - Heap invariant checker (Section 2, block states and Fig. 2; Section 3
 *     container consistency).
 *   - SMMO applications over a trivial allocator (Section 1.1, Fig. 6):
 *     game-of-life, wa-tor, n-body with merging collisions (FP64), traffic
 *     (Nagel-Schreckenberg), sugarscape (Epstein-Axtell rules M, G, R).
 *
 * Parity status: every function here is pinned by tests under tests/ against
 * closed forms, published values, invariants or brute force, except where a
 * function header says "parity unpinned".
 */
#ifndef DSR_ORACLE_H
#define DSR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- counter-based generator ------------------------------------------ */
uint64_t orc_mix64(uint64_t z);                    /* SplitMix64 finalizer */
uint64_t orc_splitmix_at(uint64_t s, uint64_t n);  /* n-th output (0-based) of SplitMix64 seeded with s */
uint64_t orc_rand(uint64_t seed, uint64_t stream, uint64_t step, uint64_t cell);
uint64_t orc_obj_hash(uint32_t type_id, const uint32_t* words, int n_words);

/* ---- hierarchical bitmap (sequential model) ---------------------------- */
typedef struct orc_hb orc_hb;
orc_hb*  orc_hb_create(uint64_t n_bits, int width, int all_set);
void     orc_hb_destroy(orc_hb* h);
int      orc_hb_levels(const orc_hb* h);
uint64_t orc_hb_level_bits(const orc_hb* h, int level);
int      orc_hb_get(const orc_hb* h, int level, uint64_t pos);
/* trace receives (level, position) pairs of every bit this call changed, in
 * order; *n_trace is the number of pairs. */
int      orc_hb_try_clear(orc_hb* h, uint64_t pos, int64_t* trace, int* n_trace);
int      orc_hb_try_set(orc_hb* h, uint64_t pos, int64_t* trace, int* n_trace);
int64_t  orc_hb_try_find_set(const orc_hb* h);     /* -1 = FAIL */
int64_t  orc_hb_clear_any(orc_hb* h);              /* find a set bit and clear it; -1 = FAIL */
int      orc_hb_consistent(const orc_hb* h);       /* 1 iff container consistency holds on every level */

/* ---- heap invariant checker --------------------------------------------
 * Bitmaps use 64-bit containers. Each bitmap over M bits is given as the
 * concatenation of its levels (level 0 first); level l has
 * words_per_level[l] words. alloc_bm / active_bm hold n_types such bitmaps
 * back to back. obj_free[b] has bit s set iff slot s of block b is free.
 * Returns a bit set of violated invariants (0 = all hold):
 *   1  I1 container consistency of some level of some bitmap
 *   2  I5 a block is in not exactly one of {free, allocated[T] for one T}
 *   4  I3 allocated[T] block whose type is not T or that holds no object
 *   8  I4 active[T] differs from "allocated[T] and has a free slot"
 *  16  a set bit outside [0, M) or a free-slot bit outside [0, capacity)
 * live_out[T] receives the number of live objects of type T (I7).
 */
uint32_t orc_check_heap(uint64_t M, int n_types, const uint32_t* capacity,
                        const uint64_t* obj_free, const uint8_t* block_type,
                        const uint64_t* free_bm, const uint64_t* alloc_bm,
                        const uint64_t* active_bm, const uint64_t* words_per_level,
                        int n_levels, int width, uint64_t* live_out);

/* ---- game of life (B3/S23 as an SMMO program) -------------------------- */
typedef struct orc_gol orc_gol;
orc_gol* orc_gol_create(int W, int H, const uint8_t* alive0);
void     orc_gol_destroy(orc_gol* g);
void     orc_gol_step(orc_gol* g, int n_gen);
int64_t  orc_gol_alive_count(const orc_gol* g);
void     orc_gol_hash(const orc_gol* g, uint64_t* cell_hash, uint64_t* alive_hash);
/* cells_out[W*H*3]: (alive, count, idx) in idx order; alive_out[cap*2]:
 * (x, y) sorted lexicographically. Returns the number of Alive objects. */
int64_t  orc_gol_dump(const orc_gol* g, int32_t* cells_out, int32_t* alive_out, int64_t cap);

/* ---- wa-tor ------------------------------------------------------------- */
typedef struct {
    int32_t W, H;
    uint64_t seed;
    int32_t fish_breed;      /* 3  */
    int32_t shark_breed;     /* 10 */
    int32_t shark_energy0;   /* 5  */
    int32_t shark_gain;      /* 3  */
} orc_wator_params;
typedef struct orc_wator orc_wator;
/* kind0[W*H]: 0 empty, 1 fish, 2 shark. */
orc_wator* orc_wator_create(const orc_wator_params* p, const uint8_t* kind0);
void       orc_wator_destroy(orc_wator* w);
/* events_out (may be NULL) receives, per step, 6 counts: fish births, fish
 * eaten, shark births, sharks starved, fish moves, shark moves. */
void       orc_wator_step(orc_wator* w, int n_steps, int64_t* events_out);
void       orc_wator_counts(const orc_wator* w, int64_t* n_fish, int64_t* n_shark);
void       orc_wator_hash(const orc_wator* w, uint64_t* fish_hash, uint64_t* shark_hash);
/* fish_out[cap*3]: (x, y, timer); shark_out[cap*4]: (x, y, timer, energy);
 * both sorted lexicographically. Returns 0, or -1 if cap is too small. */
int        orc_wator_dump(const orc_wator* w, int32_t* fish_out, int64_t fish_cap,
                          int32_t* shark_out, int64_t shark_cap);
/* kind_out[W*H] as kind0. */
void       orc_wator_grid(const orc_wator* w, uint8_t* kind_out);

/* ---- n-body with merging collisions (FP64) -----------------------------
 * orc_set_threads splits the independent per-body rows of a step across
 * threads; results are identical for every thread count. */
void       orc_set_threads(int n);
typedef struct {
    double G, eps, dt, r_merge;
} orc_nbody_params;
typedef struct orc_nbody orc_nbody;
/* body rows: (x, y, z, vx, vy, vz, m); body i gets id i. */
orc_nbody* orc_nbody_create(const orc_nbody_params* p, const double* bodies, int64_t n);
void       orc_nbody_destroy(orc_nbody* b);
/* merges_out (may be NULL): per merge (step, survivor id, absorbed id), up
 * to merges_cap merges; returns the number of merges in these steps.
 * marginal_out (may be NULL) receives the number of pairs whose distance
 * lies within `margin` of r_merge at any merge test of these steps. */
int64_t    orc_nbody_step(orc_nbody* b, int n_steps, int64_t* merges_out, int64_t merges_cap,
                          double margin, int64_t* marginal_out);
int64_t    orc_nbody_count(const orc_nbody* b);
/* rows (id, x, y, z, vx, vy, vz, m) sorted by id; returns the count. */
int64_t    orc_nbody_dump(const orc_nbody* b, double* out, int64_t cap);

/* ---- traffic (Nagel-Schreckenberg; rules in orc_traffic.cpp) ----------- */
typedef struct {
    int32_t R, L;         /* roads, cells per road */
    int32_t vmax;         /* maximum velocity (cells per step) */
    int32_t v_entry;      /* velocity of a car entering an open road */
    int32_t periodic;     /* 1: ring roads (no sources); 0: open roads */
    int32_t pad_;
    uint64_t seed;
    uint64_t p_thr;       /* dawdle iff (r >> 32) < p_thr; floor(p * 2^32) */
    uint64_t a_thr;       /* entry iff (r >> 32) < a_thr; floor(alpha * 2^32) */
} orc_traffic_params;
typedef struct orc_traffic orc_traffic;
/* v0[R*L]: -1 = empty cell, else the initial velocity of the car there. */
orc_traffic* orc_traffic_create(const orc_traffic_params* p, const int8_t* v0);
void         orc_traffic_destroy(orc_traffic* t);
/* events_out (may be NULL) receives, per step, 4 counts: cars entered, cars
 * that left, cars that moved (v > 0), and the sum of the new velocities (all
 * cars of the step, leaving ones included). */
void         orc_traffic_step(orc_traffic* t, int n_steps, int64_t* events_out);
int64_t      orc_traffic_count(const orc_traffic* t);
void         orc_traffic_hash(const orc_traffic* t, uint64_t* car_hash, uint64_t* source_hash);
/* cars_out[cap*3]: (road, x, v) sorted lexicographically; sources_out (may be
 * NULL) [R*3]: (road, entered, blocked) by road (open roads). Returns the
 * number of cars, or -1 if cap is too small. */
int64_t      orc_traffic_dump(const orc_traffic* t, int32_t* cars_out, int64_t cap, int32_t* sources_out);

/* ---- sugarscape (rules in orc_sugarscape.cpp) -------------------------- */
typedef struct {
    int32_t W, H;
    uint64_t seed;
    int32_t alpha;                   /* growback per step */
    int32_t endow_lo, endow_hi;      /* initial sugar of a new agent */
    int32_t metab_lo, metab_hi;
    int32_t vision_lo, vision_hi;    /* W, H >= 2 * vision_hi + 1 */
    int32_t age_lo, age_hi;          /* maximum age */
} orc_sugarscape_params;
typedef struct orc_sugarscape orc_sugarscape;
/* cap[W*H] in {0..4}; agents0[n][7] = (x, y, sugar, metabolism, vision, age,
 * max_age), at distinct cells. */
orc_sugarscape* orc_sugarscape_create(const orc_sugarscape_params* p, const uint8_t* cap,
                                      const int32_t* agents0, int64_t n_agents);
void            orc_sugarscape_destroy(orc_sugarscape* s);
/* events_out (may be NULL) receives, per step, 5 counts: moves, agents
 * starved, agents that reached their maximum age, replacements placed away
 * from the dead agent's cell, and the sugar harvested. */
void            orc_sugarscape_step(orc_sugarscape* s, int n_steps, int64_t* events_out);
int64_t         orc_sugarscape_count(const orc_sugarscape* s);
uint64_t        orc_sugarscape_hash(const orc_sugarscape* s);
/* agents_out[cap*8] (x, y, sugar, metabolism, vision, age, max_age, dead)
 * sorted; sugar_out (may be NULL) [W*H] the sugar of every cell. Returns the
 * number of agents, or -1 if cap is too small. */
int64_t         orc_sugarscape_dump(const orc_sugarscape* s, int32_t* agents_out, int64_t cap, int32_t* sugar_out);

#ifdef __cplusplus
}
#endif
#endif
