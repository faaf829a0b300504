/*
 * dsr_device.cuh -- device-side API of the GB300 SOA object heap.
 *
 * Include from CUDA code that allocates or deletes objects inside kernels, or
 * that defines do-all methods. Everything here runs on the device; all
 * operations are lock-free with bounded retries: a retry loop that reaches
 * its limit sets a sticky error bit in the heap and gives up, it never spins
 * forever (the paper's Alg. 1 loops forever when the heap is full; this one
 * returns DSR_NULL and sets DSR_ERR_OOM).
 *
 * Data structures (Section 2 "Block States", Section 3):
 *   obj[b]        64-bit object allocation bitmap of block b; bit s is SET
 *                 when slot s is FREE, bits at or beyond the capacity are 0.
 *                 It is the single source of truth (Section 2, linearization
 *                 point): every slot is taken and returned by an atomic on it.
 *   btype[b]      type of the objects in block b.
 *   free_bm, alloc_bm[T], active_bm[T]
 *                 hierarchical bitmaps over the M blocks (64-bit containers;
 *                 a nested bit is set iff its container is non-zero). They are
 *                 hints that are eventually consistent with obj[]: each
 *                 zero/non-zero transition of an obj[b] word obliges the
 *                 thread that caused it to set or clear the matching
 *                 active_bm bit, and set/clear retry until this thread's own
 *                 atomic changed the bit (Section 2.1), so that the bits end
 *                 up consistent once all operations have finished (Section 3).
 *
 * Handles: dsr_ref = (block << 6) | slot; DSR_NULL = all ones.
 */
#ifndef DSR_DEVICE_CUH
#define DSR_DEVICE_CUH

#include <stdint.h>

#include "dsr.h"

typedef unsigned long long dsr_u64;
typedef dsr_u64 dsr_ref;
#define DSR_NULL (~0ull)
#ifndef DSR_SPIN_CAP
#define DSR_SPIN_CAP (1u << 16)  /* set/clear retries before DSR_ERR_RETRY (about 70 ms with backoff) */
#endif
#ifndef DSR_FIND_CAP
#define DSR_FIND_CAP 4096u       /* find-and-clear attempts */
#endif
#ifndef DSR_ALLOC_CAP
#define DSR_ALLOC_CAP 4096u      /* allocation attempts before DSR_ERR_RETRY */
#endif
#define DSR_CTR_SLOTS 256u       /* event-counter rows (indexed by SM id) */
#define DSR_SLOW_WAITS 64u       /* rounds a leader may wait for another initialisation */
#define DSR_CHASE_ROUNDS 4       /* atomics on one block per search before searching again */
#ifndef DSR_FRESH_REST
#define DSR_FRESH_REST 12        /* slots still wanted after a first round that send a leader to a fresh block */
#endif

/* One hierarchical bitmap: level l has nwords[l] 64-bit containers, of
 * which the low 2^shift bits are used (the fan-out: 64, 32 or 16). */
struct dsr_hbm {
    dsr_u64* lvl[DSR_MAX_LEVELS];
    uint32_t nwords[DSR_MAX_LEVELS];
    int32_t n_levels;
    uint32_t shift;
};

/* Device view of a heap; passed by value to kernels. */
struct dsr_dev_heap {
    uint8_t* data;        /* M * block_bytes of SOA data */
    dsr_u64* obj;         /* [M] free-slot bitmaps */
    uint8_t* btype;       /* [M] */
    uint32_t* err;        /* sticky DSR_ERR_* bits */
    uint32_t* inject;     /* slow-path allocations left to fail (fault injection) */
    uint32_t* R_bid;      /* do-all block list: block ids */
    dsr_u64* R_mask;      /* do-all block list: occupied-slot snapshot */
    uint32_t* R_count;    /* entries in R (zero between do-alls) */
    uint32_t* R_done;     /* CTAs of the current method kernel that finished */
    dsr_u64* ctr;         /* [DSR_CTR_SLOTS][DSR_CTR_COUNT] event counters, one row per SM */
    uint32_t* slow;       /* [DSR_MAX_TYPES] slow-path block initialisations in flight */
    dsr_u64* dbg;         /* first failed device check (code << 48 | value), checked builds only */
    uint32_t slow_max;    /* at most this many in flight per type before leaders wait */
    dsr_u64 M;
    uint32_t block_bytes;
    int32_t n_types;
    dsr_hbm free_bm;
    dsr_hbm alloc_bm[DSR_MAX_TYPES];
    dsr_hbm active_bm[DSR_MAX_TYPES];
    dsr_u64 valid[DSR_MAX_TYPES];                  /* mask of the slots a block of type T has */
    uint32_t cap[DSR_MAX_TYPES];
    uint32_t n_fields[DSR_MAX_TYPES];
    uint32_t foff[DSR_MAX_TYPES][DSR_MAX_FIELDS];  /* byte offset of a field's SOA array */
    uint8_t fsize[DSR_MAX_TYPES][DSR_MAX_FIELDS];
    uint32_t sub[DSR_MAX_TYPES];                   /* types a do-all over T visits: T and its subtypes (bit mask) */
    uint8_t span_sh[DSR_MAX_TYPES];                /* log2 threads per listed block in a do-all over T */
};

#ifdef __CUDACC__

/* ------------------------------------------------------------------------ */
/* small helpers                                                            */
/* ------------------------------------------------------------------------ */
__device__ __forceinline__ dsr_u64 dsr_ld_relaxed(const dsr_u64* p) {
    dsr_u64 v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

/* 64-bit atomics with acquire or release ordering (PTX memory model), used
 * where a block's object bitmap publishes or guards its type byte. The
 * atomics that take a block's slots (reserve) or lock an empty block
 * (reclaim) need only acquire: the type read and the bitmap updates that
 * follow them must not be performed before them, while nothing before them
 * is published through them. Acquire without release spares the memory
 * barrier ahead of the atomic, which an allocation would wait on. */
__device__ __forceinline__ dsr_u64 dsr_atom_and_acquire(dsr_u64* p, dsr_u64 v) {
    dsr_u64 old;
    asm volatile("atom.acquire.gpu.global.and.b64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ dsr_u64 dsr_atom_cas_acquire(dsr_u64* p, dsr_u64 cmp, dsr_u64 v) {
    dsr_u64 old;
    asm volatile("atom.acquire.gpu.global.cas.b64 %0, [%1], %2, %3;" : "=l"(old) : "l"(p), "l"(cmp), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ void dsr_atom_exch_release(dsr_u64* p, dsr_u64 v) {
    [[maybe_unused]] dsr_u64 old;  // the exchange's result is not needed
    asm volatile("atom.release.gpu.global.exch.b64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
}

/* Device self-checks, compiled in with -DDSR_DEVICE_CHECKS: a failed check
 * sets DSR_ERR_CHECK, records the first failure (code << 48 | value) and
 * returns false so that the caller skips the access. Without the macro every
 * check is true and costs nothing. */
#define DSR_ERR_CHECK 32u
__device__ __forceinline__ bool dsr_check(bool ok, uint32_t* err, dsr_u64* dbg, unsigned code, dsr_u64 value) {
#ifdef DSR_DEVICE_CHECKS
    if (!ok) {
        atomicOr(err, DSR_ERR_CHECK);
        atomicCAS(dbg, 0ull, ((dsr_u64)code << 48) | (value & 0xFFFFFFFFFFFFull));
        return false;
    }
    return true;
#else
    (void)ok;
    (void)err;
    (void)dbg;
    (void)code;
    (void)value;
    return true;
#endif
}

__device__ __forceinline__ unsigned dsr_lane() {
    unsigned l;
    asm("mov.u32 %0, %%laneid;" : "=r"(l));
    return l;
}

/* Add n to event counter k (DSR_CTR_*) in the row of the calling SM, so that
 * warps of different SMs never contend on one address. */
__device__ __forceinline__ void dsr_count(dsr_u64* ctr, unsigned k, dsr_u64 n) {
    unsigned smid;
    asm("mov.u32 %0, %%smid;" : "=r"(smid));
    atomicAdd(ctr + (smid % DSR_CTR_SLOTS) * DSR_CTR_COUNT + k, n);
}

/* Count one event per calling lane: one atomic per warp and heap. */
__device__ __forceinline__ void dsr_count_lanes(dsr_u64* ctr, unsigned k) {
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, (dsr_u64)reinterpret_cast<uintptr_t>(ctr));
    if (dsr_lane() == (unsigned)(__ffs(peers) - 1)) dsr_count(ctr, k, (dsr_u64)__popc(peers));
}

__device__ __forceinline__ void dsr_backoff(unsigned tries) {
    if (tries > 8) __nanosleep(tries < 32 ? 32u * tries : 1024u);
}

/* Position of the n-th (0-based) set bit of m; requires n < popc(m). */
__device__ __forceinline__ int dsr_nth_bit(dsr_u64 m, int n) {
    int pos = 0;
#pragma unroll
    for (int w = 32; w >= 1; w >>= 1) {
        int c = __popcll(m & ((1ull << w) - 1));
        if (n >= c) {
            n -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

__device__ __forceinline__ dsr_u64 dsr_rotr(dsr_u64 m, unsigned r) { return r ? (m >> r) | (m << (64 - r)) : m; }
__device__ __forceinline__ dsr_u64 dsr_rotl(dsr_u64 m, unsigned r) { return r ? (m << r) | (m >> (64 - r)) : m; }

/* The lowest min(k, popc(m)) set bits of m. */
__device__ __forceinline__ dsr_u64 dsr_lowest_bits(dsr_u64 m, int k) {
    if (k >= __popcll(m)) return m;
    return m & ((1ull << dsr_nth_bit(m, k)) - 1);
}

/* ------------------------------------------------------------------------ */
/* hierarchical bitmap operations (Section 2.1, Alg. 2)                     */
/* ------------------------------------------------------------------------ */

/* The bitmap operations are written once over a compile-time container
 * shift SH (6: 64-bit fan-out); SH == 0 reads the shift from the bitmap at
 * run time. The public entry points take the constant-shift path for the
 * default fan-out, where 64-bit shifts by constants are single
 * instructions, and the run-time path for 32 and 16. */
template <unsigned SH>
__device__ __forceinline__ unsigned dsr_hb_shift(const dsr_hbm& b) {
    return SH ? SH : b.shift;
}

/* Set bit pos of level l. With retry == false this is try_set: it fails if
 * the bit is already set. With retry == true it is set(pos): it retries until
 * its own atomicOr changed the bit. If the container was empty before, this
 * thread owes the nested bit, which it sets with set() (never try_set). */
template <unsigned SH>
__device__ __forceinline__ bool dsr_hb_set_t(const dsr_hbm& b, dsr_u64 pos, bool retry, uint32_t* err) {
    const unsigned sh = dsr_hb_shift<SH>(b);
    const dsr_u64 lo = (1ull << sh) - 1;
    for (int l = 0; l < b.n_levels; ++l) {
        dsr_u64* w = b.lvl[l] + (pos >> sh);
        const dsr_u64 m = 1ull << (pos & lo);
        dsr_u64 prev;
        for (unsigned tries = 0;; ++tries) {
            prev = atomicOr(w, m);
            if (!(prev & m)) break;
            if (!retry) return false;
            if (tries >= DSR_SPIN_CAP) {
                atomicOr(err, DSR_ERR_RETRY);
                return false;
            }
            dsr_backoff(tries);
        }
        retry = true;
        if (prev != 0) break;  // container already non-empty: nothing owed above
        pos >>= sh;
    }
    return true;
}

/* Clear bit pos of level l (Alg. 2). try_clear when retry == false, clear(pos)
 * otherwise. If this call cleared the last set bit of its container
 * (popc(prev) == 1) it clears the nested bit with clear(). */
template <unsigned SH>
__device__ __forceinline__ bool dsr_hb_clear_t(const dsr_hbm& b, dsr_u64 pos, bool retry, uint32_t* err) {
    const unsigned sh = dsr_hb_shift<SH>(b);
    const dsr_u64 lo = (1ull << sh) - 1;
    for (int l = 0; l < b.n_levels; ++l) {
        dsr_u64* w = b.lvl[l] + (pos >> sh);
        const dsr_u64 m = 1ull << (pos & lo);
        dsr_u64 prev;
        for (unsigned tries = 0;; ++tries) {
            prev = atomicAnd(w, ~m);
            if (prev & m) break;
            if (!retry) return false;
            if (tries >= DSR_SPIN_CAP) {
                atomicOr(err, DSR_ERR_RETRY);
                return false;
            }
            dsr_backoff(tries);
        }
        retry = true;
        if (prev != m) break;  // other bits remain in the container
        pos >>= sh;
    }
    return true;
}

__device__ __forceinline__ bool dsr_hb_set(const dsr_hbm& b, dsr_u64 pos, bool retry, uint32_t* err) {
    return b.shift == 6 ? dsr_hb_set_t<6>(b, pos, retry, err) : dsr_hb_set_t<0>(b, pos, retry, err);
}
__device__ __forceinline__ bool dsr_hb_clear(const dsr_hbm& b, dsr_u64 pos, bool retry, uint32_t* err) {
    return b.shift == 6 ? dsr_hb_clear_t<6>(b, pos, retry, err) : dsr_hb_clear_t<0>(b, pos, retry, err);
}

/* 32-bit integer hash (the "lowbias32" finalizer published by C. Wellons,
 * 2018): spreads consecutive or similar hints over all 32 bits. */
__device__ __forceinline__ unsigned dsr_hash32(unsigned x) {
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x;
}

/* try_find_set (Section 2.1, Section 2.4): descend from the top level, one
 * container read per level. At each level the searcher takes one of the
 * container's set bits, chosen uniformly by a hash of (hint, level), so that
 * concurrent searchers with different hints spread evenly over the set bits
 * (a "first set bit after an offset" rule would favour bits that follow long
 * runs of zeros, and the first bit of a container whose high bits are zero).
 * Returns -1 (FAIL) if a container on the way is empty, which can happen
 * while the bitmap is temporarily inconsistent. */
/* The descent is preceded by a shortcut: one leaf container, drawn from the
 * hint, is read together with the top-level container (two independent
 * loads). If that leaf has a set bit, the search ends after one round trip
 * instead of one per level; this is the common case when most leaves are
 * non-empty (an allocator whose blocks of a type mostly have free slots).
 * Otherwise the descent continues from the top-level word already read. */
template <unsigned SH>
__device__ __forceinline__ long long dsr_hb_find_t(const dsr_hbm& b, unsigned hint) {
    const unsigned sh = dsr_hb_shift<SH>(b);
    const int top = b.n_levels - 1;
    const unsigned hp = dsr_hash32(hint ^ 0x5851F42Du);
    const dsr_u64 li = __umulhi(hp, b.nwords[0]);
    const dsr_u64 lw = dsr_ld_relaxed(b.lvl[0] + li);
    dsr_u64 w = dsr_ld_relaxed(b.lvl[top]);
    if (lw != 0) return (long long)((li << sh) + (dsr_u64)dsr_nth_bit(lw, (int)__umulhi(dsr_hash32(hp), (unsigned)__popcll(lw))));
    dsr_u64 pos = 0;
    for (int l = top; l >= 0; --l) {
        if (l != top) w = dsr_ld_relaxed(b.lvl[l] + pos);
        if (w == 0) return -1;
        const unsigned h = dsr_hash32(hint ^ ((unsigned)l * 0x9E3779B9u));
        const int k = dsr_nth_bit(w, (int)__umulhi(h, (unsigned)__popcll(w)));
        pos = (pos << sh) + (dsr_u64)k;
    }
    return (long long)pos;
}
__device__ __forceinline__ long long dsr_hb_find(const dsr_hbm& b, unsigned hint) {
    return b.shift == 6 ? dsr_hb_find_t<6>(b, hint) : dsr_hb_find_t<0>(b, hint);
}

/* clear() of Section 2.1: find a set bit and clear it. The printed loop is
 * read as: repeat { i = try_find_set(); if FAIL give up; if try_clear(i)
 * return i }, with a bounded number of rounds, and FAIL reported only after
 * the top-level container reads empty or the rounds run out. */
__device__ __forceinline__ long long dsr_hb_clear_any(const dsr_hbm& b, unsigned hint, uint32_t* err) {
    for (unsigned a = 0; a < DSR_FIND_CAP; ++a) {
        const long long i = dsr_hb_find(b, hint + a * 0x9E3779B9u);
        if (i < 0) {
            if (dsr_ld_relaxed(b.lvl[b.n_levels - 1]) == 0) return -1;
            dsr_backoff(a);
            continue;
        }
        if (dsr_hb_clear(b, (dsr_u64)i, false, err)) return i;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* block-level allocation and release                                      */
/* ------------------------------------------------------------------------ */
struct dsr_grab {
    dsr_u64 bid;
    dsr_u64 bits;     /* slots taken (their free bits were cleared by this call) */
    uint32_t status;  /* 0 or a DSR_ERR_* bit */
};

__device__ __forceinline__ int dsr_block_type(const dsr_dev_heap& H, dsr_u64 b) {
    return *(volatile const uint8_t*)(H.btype + b);
}

/* Return the slots `bits` of block b (type T) to the heap. The atomicOr on
 * obj[b] is the linearization point. A zero -> non-zero transition (the block
 * was full) obliges active[T].set(b). A block that became empty is reclaimed
 * by whoever wins the CAS valid -> 0 that locks it: that CAS takes every free
 * slot, so it is a non-zero -> zero transition that obliges
 * active[T].clear(b); then allocated[T].clear(b) and free.set(b). The type is
 * re-read after the CAS: if the block was reclaimed and reused meanwhile, the
 * CAS either fails or takes the free slots of the reused block, which are
 * then returned through this same path. Deallocation is not spelled out in
 * the paper's abstract; this protocol is this library's reading of the block
 * states of Fig. 2 and the linearization rule of Section 2. */
__device__ inline void dsr_release(const dsr_dev_heap& H, int T, dsr_u64 b, dsr_u64 bits) {
    for (int round = 0; round < 4 && bits; ++round) {
        const dsr_u64 prev = atomicOr(H.obj + b, bits);
        if (prev & bits) {
            atomicOr(H.err, DSR_ERR_DOUBLE_FREE);
            bits &= ~prev;
            if (!bits) return;
        }
        if (prev == 0) dsr_hb_set(H.active_bm[T], b, true, H.err);
        const dsr_u64 v = H.valid[T];
        if ((prev | bits) != v) return;
        if (dsr_atom_cas_acquire(H.obj + b, v, 0ull) != v) return;
        const int T2 = dsr_block_type(H, b);  // ordered after the acquiring CAS
        dsr_hb_clear(H.active_bm[T2], b, true, H.err);
        if (H.valid[T2] == v) {
            dsr_hb_clear(H.alloc_bm[T2], b, true, H.err);
            dsr_hb_set(H.free_bm, b, true, H.err);
            return;
        }
        // The CAS took the free slots of a reused, non-empty block of another
        // type: give them back.
        T = T2;
        bits = v;
    }
}

/* Slow path of Alg. 1: take a block from the free bitmap (find and clear),
 * initialise it for T with its first min(k, capacity) slots already taken,
 * publish its object bitmap, then set allocated[T] and, if slots remain,
 * active[T]. status DSR_ERR_OOM: fault injection; DSR_ERR_RETRY: no free
 * block was found. */
__device__ inline dsr_grab dsr_init_block(const dsr_dev_heap& H, int T, int k, unsigned hint) {
    if (H.inject && *(volatile uint32_t*)H.inject != 0) {
        const unsigned v = atomicSub(H.inject, 1u);
        if (v != 0 && v < 0x80000000u) return {0, 0, DSR_ERR_OOM};
        atomicAdd(H.inject, 1u);  // the count ran out under us: undo
    }
    const long long b = dsr_hb_clear_any(H.free_bm, hint, H.err);
    if (b < 0) return {0, 0, DSR_ERR_RETRY};
    const unsigned c = H.cap[T];
    const unsigned take = (unsigned)k < c ? (unsigned)k : c;
    const dsr_u64 want = take >= 64 ? ~0ull : ((1ull << take) - 1);
    const dsr_u64 rest = H.valid[T] & ~want;
    H.btype[b] = (uint8_t)T;
    dsr_atom_exch_release(H.obj + b, rest);  // publishes the type with the bitmap
    dsr_count(H.ctr, DSR_CTR_BLOCKS, 1);
    dsr_hb_set(H.alloc_bm[T], (dsr_u64)b, true, H.err);
    if (rest) dsr_hb_set(H.active_bm[T], (dsr_u64)b, true, H.err);
    return {(dsr_u64)b, want, 0};
}

/* Alg. 1 for up to k objects of type T, run by one thread (the leader of a
 * warp's requests for T, Section 2.4). Fast path: find a block in active[T],
 * take the lowest free slots of a snapshot of its bitmap with one atomicAnd,
 * keep those actually obtained; if that emptied the free bits, clear
 * active[T] (the block is full). Slow path: take a block from free (find and
 * clear), initialise it for T with the first slots already taken, publish
 * its bitmap, then set allocated[T] and, if slots remain, active[T]. With
 * `fresh` the first attempt goes to the slow path directly; when the
 * throttle holds it back or no free block is left, the fast path follows as
 * usual, so a heap whose only free slots are in active blocks still serves
 * the request. With near_block >= 0 (a block of this heap) the first
 * attempt takes that block instead of a search: its free-slot word is read
 * and the slots are taken as from a found block; a full block, one of
 * another type or one being reclaimed gives nothing and the search
 * follows. */
__device__ inline dsr_grab dsr_reserve(const dsr_dev_heap& H, int T, int k, unsigned hint, bool fresh = false,
                                       long long near_block = -1) {
    unsigned empty_rounds = 0;  // slow paths that found no free block
    for (unsigned a = 0; a < DSR_ALLOC_CAP; ++a) {
        long long b = a == 0 && near_block >= 0 ? near_block
                      : fresh && a == 0       ? -1
                                              : dsr_hb_find(H.active_bm[T], hint + a * 0x61C88647u);
        if (b < 0) {
            // Many warps miss the fast path at the same moment (a kernel that
            // starts by allocating). Rather than each opening its own block,
            // which would leave thousands of blocks nearly empty, at most
            // slow_max leaders per type initialise blocks at a time; the
            // others wait briefly and retry the fast path on the blocks just
            // published. After DSR_SLOW_WAITS rounds a leader goes ahead.
            bool counted = false;
            if (a < DSR_SLOW_WAITS) {
                if (*(volatile uint32_t*)(H.slow + T) >= H.slow_max) {
                    dsr_backoff(a + 12);
                    continue;
                }
                if (atomicAdd(H.slow + T, 1u) >= H.slow_max) {
                    atomicSub(H.slow + T, 1u);
                    dsr_backoff(a + 12);
                    continue;
                }
                counted = true;
            }
            const dsr_grab g = dsr_init_block(H, T, k, hint ^ (a * 0x9E3779B9u));
            if (counted) atomicSub(H.slow + T, 1u);
            if (g.status == 0) return g;
            // No free block (or an injected failure). Slots may still be in
            // flight: a block another leader just initialised, or a release
            // between its slot return and its active[T].set. Retry the fast
            // path a few times before reporting out-of-memory.
            if (g.status != DSR_ERR_RETRY || ++empty_rounds >= 16) return {0, 0, DSR_ERR_OOM};
            dsr_backoff(empty_rounds + 9);
            continue;
        }
        // Take free slots of a snapshot, the first ones at or after a slot
        // offset drawn from the hint (leaders that meet on one block then
        // mostly ask for different slots); while the block still has free
        // slots (as the atomic's return value shows) and more are wanted,
        // take those too, for a few rounds, without searching again.
        dsr_u64* w = H.obj + b;
        dsr_u64 snap = dsr_ld_relaxed(w);
        if (snap == 0) {
            dsr_backoff(a);
            continue;
        }
        const unsigned rot = dsr_hash32(hint + a) >> 26;
        dsr_u64 got = 0;
        bool emptied = false;
        for (int r = 0; r < DSR_CHASE_ROUNDS && snap; ++r) {
            const dsr_u64 want = dsr_rotl(dsr_lowest_bits(dsr_rotr(snap, rot), k - __popcll(got)), rot);
            const dsr_u64 prev = dsr_atom_and_acquire(w, ~want);
            got |= prev & want;
            snap = prev & ~want;
            emptied = prev != 0 && snap == 0;  // this atomic left no free slot
            if (__popcll(got) >= k) break;
        }
        if (!got) continue;
        // The acquire above orders this read after the atomic: while this
        // call holds slots of the block, its type cannot change.
        const int T2 = dsr_block_type(H, (dsr_u64)b);
        if (emptied) dsr_hb_clear(H.active_bm[T2], (dsr_u64)b, true, H.err);
        if (T2 != T) {
            // Stale hint: the block was reclaimed and reused for another type.
            dsr_release(H, T2, (dsr_u64)b, got);
            continue;
        }
        return {(dsr_u64)b, got, 0};
    }
    return {0, 0, DSR_ERR_RETRY};
}

/* ------------------------------------------------------------------------ */
/* public device API                                                         */
/* ------------------------------------------------------------------------ */

/* Key that identifies a heap among the lanes of a warp: the address of its
 * object bitmaps (256-byte aligned, so the low bits are free for a type id).
 * Lanes that meet at one call site may come from different iterations of a
 * kernel's loop (independent thread scheduling lets them drift apart and
 * converge again) and so may work on different heaps; aggregation must only
 * combine lanes of the same heap. */
__device__ __forceinline__ dsr_u64 dsr_heap_key(const dsr_dev_heap& H) {
    return (dsr_u64)reinterpret_cast<uintptr_t>(H.obj);
}

/* new T: callable by any subset of a warp's lanes, with any mix of heaps and
 * types. Lanes asking for the same type of the same heap are served by one
 * leader (allocation request coalescing, Section 2.4): it reserves slots for
 * all of them, in as few atomics as the free slots allow, and hands them out
 * by shuffle. Returns DSR_NULL (and sets DSR_ERR_OOM or DSR_ERR_RETRY) on
 * failure. The new object's fields are not initialised. `near` (optional):
 * an object of the same heap whose block the leader tries first, before
 * searching the bitmaps (the leader's own hint counts for its group), for
 * example the parent of a newborn or an object just deleted; a hint only,
 * any handle of the heap or DSR_NULL is allowed. */
__device__ inline dsr_ref dsr_new(const dsr_dev_heap& H, int T, dsr_ref near = DSR_NULL) {
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, dsr_heap_key(H) | (dsr_u64)T);
    const unsigned lane = dsr_lane();
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1));
    const int need = __popc(peers);
    const unsigned hint = (blockIdx.x * 0x9E3779B1u) ^ ((threadIdx.x >> 5) * 0x85EBCA77u) ^ (unsigned)T;
    dsr_ref mine = DSR_NULL;
    int served = 0;
    // Each round the leader takes as many slots as the block it finds (or a
    // new block) offers, until the group is served.
    int round = 0;  // reservation rounds of the leader
    while (served < need) {
        dsr_u64 bid = 0, bits = 0;
        uint32_t st = 0;
        if ((int)lane == leader) {
            // The first round tries the leader's placement hint, if it gave
            // one. A group still wanting many slots after a round that
            // searched takes a fresh block rather than walking partly
            // filled ones one by one.
            const long long nb = round == 0 && near != DSR_NULL && (near >> 6) < H.M ? (long long)(near >> 6) : -1;
            const bool fresh = DSR_FRESH_REST > 0 && served > 0 && round > (near != DSR_NULL ? 1 : 0) &&
                               need - served >= DSR_FRESH_REST;
            const dsr_grab g = dsr_reserve(H, T, need - served, hint + (unsigned)served, fresh, nb);
            bid = g.bid;
            bits = g.bits;
            st = g.status;
            if (st) atomicOr(H.err, st);
            else dsr_count(H.ctr, DSR_CTR_ALLOCS, (dsr_u64)__popcll(bits));
        }
        bid = __shfl_sync(peers, bid, leader);
        bits = __shfl_sync(peers, bits, leader);
        st = __shfl_sync(peers, st, leader);
        if (st) break;
        const int n = __popcll(bits);
        if (rank >= served && rank < served + n) mine = (bid << 6) | (dsr_u64)dsr_nth_bit(bits, rank - served);
        served += n;
        ++round;
    }
    return mine;
}

/* delete: callable by any subset of a warp's lanes, with any mix of heaps.
 * Lanes deleting objects of the same block of the same heap are combined
 * into one atomicOr by a leader. DSR_NULL is ignored; a handle outside the
 * heap sets DSR_ERR_BAD_HANDLE. */
__device__ inline void dsr_delete(const dsr_dev_heap& H, dsr_ref r) {
    if (r == DSR_NULL) return;
    const unsigned act = __activemask();
    const dsr_u64 bid = r >> 6;
    const unsigned slot = (unsigned)(r & 63);
    const unsigned peers = __match_any_sync(act, bid) & __match_any_sync(act, dsr_heap_key(H));
    const unsigned lane = dsr_lane();
    const unsigned lo = __reduce_or_sync(peers, slot < 32 ? (1u << slot) : 0u);
    const unsigned hi = __reduce_or_sync(peers, slot >= 32 ? (1u << (slot - 32)) : 0u);
    if ((int)lane != __ffs(peers) - 1) return;
    if (bid >= H.M) {
        atomicOr(H.err, DSR_ERR_BAD_HANDLE);
        return;
    }
    const int T = dsr_block_type(H, bid);
    if (T >= H.n_types) {
        atomicOr(H.err, DSR_ERR_BAD_HANDLE);
        return;
    }
    dsr_u64 bits = ((dsr_u64)hi << 32) | lo;
    if (bits & ~H.valid[T]) {  // a slot at or beyond the block's capacity
        atomicOr(H.err, DSR_ERR_BAD_HANDLE);
        bits &= H.valid[T];
        if (!bits) return;
    }
    dsr_count(H.ctr, DSR_CTR_FREES, (dsr_u64)__popcll(bits));
    dsr_release(H, T, bid, bits);
}

/* Address of field f of the object r (type T): block base + the field's SOA
 * array offset + slot * field size. Consecutive slots are adjacent. */
template <class F>
__device__ __forceinline__ F* dsr_field(const dsr_dev_heap& H, int T, dsr_ref r, int f) {
#ifdef DSR_DEVICE_CHECKS
    // a bad handle is redirected to scratch words next to the check record
    if (!dsr_check((r >> 6) < H.M && (r & 63) < H.cap[T], H.err, H.dbg, 11, r))
        return reinterpret_cast<F*>(H.dbg + 1);
#endif
    return reinterpret_cast<F*>(H.data + (r >> 6) * H.block_bytes + H.foff[T][f]) + (r & 63);
}

/* ------------------------------------------------------------------------ */
/* parallel do-all (Section 2.3)                                           */
/* ------------------------------------------------------------------------ */

/* Threads per listed block in the method kernel: 32 when the capacity of
 * every type the do-all visits fits one warp, else 64. Each warp then covers
 * one block, reads its R entry once and touches one contiguous segment of
 * every SOA array. */
__device__ __forceinline__ unsigned dsr_span_shift(const dsr_dev_heap& H, int T) { return H.span_sh[T]; }

/* Concrete type of a listed block in a do-all over T: T itself, unless T has
 * subtypes (dsr_heap_set_bases), whose blocks the list may also hold; then
 * the block's type byte. */
__device__ __forceinline__ int dsr_listed_type(const dsr_dev_heap& H, int T, uint32_t bid) {
    return H.sub[T] == (1u << T) ? T : (int)H.btype[bid];
}

/* End of every kernel that consumes R: the last CTA to finish resets the
 * block-list counter for the next do-all. Returns true in thread 0 of that
 * last CTA. */
__device__ __forceinline__ bool dsr_doall_finish(const dsr_dev_heap& H, bool keep_list = false) {
    __syncthreads();
    bool last = false;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(H.R_done, 1u);
        if (t == gridDim.x - 1) {
            if (!keep_list) *(volatile uint32_t*)H.R_count = 0;
            *(volatile uint32_t*)H.R_done = 0;
            __threadfence();
            last = true;
        }
    }
    return last;
}

/* Optional end-of-do-all hook: Method::finish(H, T, args) runs once, in the
 * last CTA, after every object has been visited. */
template <class M>
__device__ __forceinline__ auto dsr_call_finish(const dsr_dev_heap& H, int T, const typename M::Args& a, int)
    -> decltype(M::finish(H, T, a), void()) {
    M::finish(H, T, a);
}
template <class M>
__device__ __forceinline__ void dsr_call_finish(const dsr_dev_heap&, int, const typename M::Args&, long) {}

/* Method kernel of a do-all over type T. Method is a type with
 *   struct Args;  (trivially copyable)
 *   static __device__ void run(const dsr_dev_heap&, int T, const Args&, dsr_ref self);
 *   optionally static __device__ void finish(const dsr_dev_heap&, int T, const Args&);
 * run gets the concrete type of `self`: T, or one of T's subtypes when the
 * heap declares them (dsr_heap_set_bases). Persistent grid-stride loop over (listed block, slot); a slot runs the
 * method iff it was occupied in the snapshot taken by the scan. With
 * keep_list the block list R survives the kernel, for a following do-all
 * over the same live set (one whose predecessor created and deleted no
 * object of T) that then skips its scan. */
template <class Method>
__device__ __forceinline__ void dsr_doall_body(const dsr_dev_heap& H, int T, const typename Method::Args& args,
                                               int keep_list) {
    const unsigned sh = dsr_span_shift(H, T);
    const dsr_u64 total = (dsr_u64)(*(volatile uint32_t*)H.R_count) << sh;
    const dsr_u64 stride = (dsr_u64)gridDim.x * blockDim.x;
    for (dsr_u64 g = (dsr_u64)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        // total and stride are multiples of 32, so every lane of a warp runs
        // the same iterations. Reconverge the warp at each one: lanes that
        // drifted apart in a method's divergent code would otherwise reach
        // dsr_new in smaller groups, and aggregation would serve fewer lanes
        // per search.
        __syncwarp();
        const dsr_u64 i = g >> sh;
        const unsigned s = (unsigned)(g & ((1u << sh) - 1));
        // i < R_count: both entries are valid, so they load together
        const dsr_u64 mask = H.R_mask[i];
        const uint32_t bid = H.R_bid[i];
        if (((mask >> s) & 1ull) && dsr_check(bid < H.M, H.err, H.dbg, 10, i))
            Method::run(H, dsr_listed_type(H, T, bid), args, ((dsr_u64)bid << 6) | s);
    }
    if (dsr_doall_finish(H, keep_list != 0)) dsr_call_finish<Method>(H, T, args, 0);
}
template <class Method>
__global__ void dsr_doall_kernel(const __grid_constant__ dsr_dev_heap H, int T,
                                 const __grid_constant__ typename Method::Args args, int keep_list = 0) {
    dsr_doall_body<Method>(H, T, args, keep_list);
}
/* The same kernel for CTAs of at most 256 threads, compiled for at least six
 * such CTAs per SM (at most 40 registers a thread). The methods are chains
 * of dependent loads and atomics: more resident warps hide more of their
 * latency. */
template <class Method>
__global__ void __launch_bounds__(256, 6) dsr_doall_kernel_256(const __grid_constant__ dsr_dev_heap H, int T,
                                                              const __grid_constant__ typename Method::Args args,
                                                              int keep_list = 0) {
    dsr_doall_body<Method>(H, T, args, keep_list);
}

/* Vector method kernel: a method may also provide
 *   static __device__ void run4(const dsr_dev_heap&, int T, const Args&,
 *                               uint32_t block, unsigned slot0, unsigned live4);
 * which handles the four slots slot0 .. slot0 + 3 of one block at once
 * (live4: which of them were occupied in the snapshot; never 0), so that
 * each thread moves 16 bytes of a field column per access. The do-all uses
 * it when every field array of T starts on a 16-byte boundary (capacity a
 * multiple of 4 for 4-byte fields); otherwise it runs `run`. A quad of
 * threads per 16 slots: a warp covers two 64-slot blocks (or four of 32). */
template <class M, class = void>
struct dsr_has_run4 {
    static constexpr bool value = false;
};
template <class M>
struct dsr_has_run4<M, decltype(M::run4(*(const dsr_dev_heap*)nullptr, 0, *(const typename M::Args*)nullptr, 0u, 0u,
                                        0u), void())> {
    static constexpr bool value = true;
};

template <class Method>
__global__ void dsr_doall_kernel_vec4(const __grid_constant__ dsr_dev_heap H, int T,
                                      const __grid_constant__ typename Method::Args args, int keep_list = 0) {
    const unsigned sh = dsr_span_shift(H, T) - 2;  // quads per listed block: 16 (or 8)
    const dsr_u64 total = (dsr_u64)(*(volatile uint32_t*)H.R_count) << sh;
    const dsr_u64 stride = (dsr_u64)gridDim.x * blockDim.x;
    for (dsr_u64 g = (dsr_u64)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        const dsr_u64 i = g >> sh;
        const unsigned q = (unsigned)(g & ((1u << sh) - 1));
        const unsigned live = (unsigned)(H.R_mask[i] >> (4 * q)) & 0xFu;
        const uint32_t bid = H.R_bid[i];
        if (live && dsr_check(bid < H.M, H.err, H.dbg, 10, i)) Method::run4(H, T, args, bid, 4 * q, live);
    }
    if (dsr_doall_finish(H, keep_list != 0)) dsr_call_finish<Method>(H, T, args, 0);
}

/* ------------------------------------------------------------------------ */
/* heap groups: one do-all over many heaps                                  */
/* ------------------------------------------------------------------------ */

/* Device view of a heap group (dsr_group_* in dsr.h): the device views of its
 * heaps, the chunk table that maps each run of 256 block ids to its heap,
 * and the group's block list R (heap index, block id, occupied-slot
 * snapshot). */
struct dsr_group_dev {
    const dsr_dev_heap* heaps;  /* [max_heaps] */
    const uint32_t* chunk_heap; /* [n_chunks] heap of each chunk */
    const uint32_t* chunk_base; /* [n_chunks] first block id of each chunk */
    uint32_t n_chunks;
    uint32_t n_slots;           /* heap indices in use are below this */
    uint32_t* R_heap;
    uint32_t* R_bid;
    dsr_u64* R_mask;
    uint32_t* R_count;
    uint32_t* R_done;
    dsr_u64 R_cap;              /* entries R can hold */
    uint32_t* err;              /* group-level check failures (checked builds) */
    dsr_u64* dbg;
};

/* Method kernel of a group do-all over type T (all heaps of a group share
 * their type descriptors and tuning, so the span is the same for all). A
 * group method is a type with
 *   struct Args;
 *   static __device__ void run(const dsr_dev_heap&, int T, const Args&, dsr_ref self, uint32_t heap);
 *   optionally static __device__ void finish_group(const dsr_group_dev&, int T, const Args&);
 * finish_group runs in every thread of the last CTA to finish, after every
 * object has been visited. */
template <class M>
__device__ __forceinline__ auto dsr_call_finish_group(const dsr_group_dev& G, int T, const typename M::Args& a, int)
    -> decltype(M::finish_group(G, T, a), void()) {
    M::finish_group(G, T, a);
}
template <class M>
__device__ __forceinline__ void dsr_call_finish_group(const dsr_group_dev&, int, const typename M::Args&, long) {}

template <class Method>
__device__ __forceinline__ void dsr_group_doall_body(const dsr_group_dev& G, int T, unsigned sh,
                                                     const typename Method::Args& args, int keep_list) {
    __shared__ bool last;
    const dsr_u64 total = (dsr_u64)(*(volatile uint32_t*)G.R_count) << sh;
    const dsr_u64 stride = (dsr_u64)gridDim.x * blockDim.x;
    for (dsr_u64 g = (dsr_u64)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        __syncwarp();  // warp-uniform loop: reconverge as in dsr_doall_kernel
        const dsr_u64 i = g >> sh;
        const unsigned s = (unsigned)(g & ((1u << sh) - 1));
        if ((G.R_mask[i] >> s) & 1ull) {
            const uint32_t h = G.R_heap[i];
            if (dsr_check(h < G.n_slots, G.err, G.dbg, 3, i) &&
                dsr_check(G.R_bid[i] < G.heaps[h].M, G.err, G.dbg, 4, i))
                Method::run(G.heaps[h], T, args, ((dsr_u64)G.R_bid[i] << 6) | s, h);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(G.R_done, 1u) == gridDim.x - 1;
        if (last) {
            if (!keep_list) *(volatile uint32_t*)G.R_count = 0;
            *(volatile uint32_t*)G.R_done = 0;
            __threadfence();
        }
    }
    __syncthreads();
    if (last) dsr_call_finish_group<Method>(G, T, args, 0);
}
template <class Method>
__global__ void dsr_group_doall_kernel(const __grid_constant__ dsr_group_dev G, int T, unsigned sh,
                                       const __grid_constant__ typename Method::Args args, int keep_list = 0) {
    dsr_group_doall_body<Method>(G, T, sh, args, keep_list);
}
/* At most 256 threads a CTA, at least six CTAs per SM, as dsr_doall_kernel_256. */
template <class Method>
__global__ void __launch_bounds__(256, 6)
    dsr_group_doall_kernel_256(const __grid_constant__ dsr_group_dev G, int T, unsigned sh,
                               const __grid_constant__ typename Method::Args args, int keep_list = 0) {
    dsr_group_doall_body<Method>(G, T, sh, args, keep_list);
}

#endif /* __CUDACC__ */
#endif /* DSR_DEVICE_CUH */
