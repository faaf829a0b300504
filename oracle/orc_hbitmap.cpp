// Oracle: hierarchical bitmap (sequential model) and heap invariant checker.
// Test infrastructure only.
//
// Hierarchical bitmap, Section 3 "Data Structure": a bitmap of N bits is a
// sequence of containers of `width` bits (the paper uses 64; its Fig. 5
// example uses 4) plus, when N > width, a nested bitmap with one bit per
// container. A nested bit is set iff some bit of its container is set
// (container-consistency equation). Levels are built until a level fits in
// one container.
//
// Operations, Section 2.1 and Alg. 2, in a single thread (no other thread can
// make the bitmap inconsistent, so the retrying forms never retry here):
//   try_clear(pos): clear bit pos; report whether it was set. If it was and it
//                   was the last set bit of its container, clear the container's
//                   bit in the nested bitmap.
//   try_set(pos):   the mirror image: if the container was empty before, set
//                   the container's bit in the nested bitmap.
//   try_find_set(): descend from the top level, at each level taking the
//                   lowest set bit of the container the level above points
//                   to; FAIL if a container on the way is empty.
//   clear():        find a set bit and clear it (the reading of the garbled
//                   loop in Section 2.1: return FAIL when nothing is found,
//                   else the position cleared).
#include "oracle.h"

#include <cstdlib>
#include <vector>

struct orc_hb {
    int width;
    std::vector<std::vector<uint8_t>> lv;  // lv[l][i] = bit i of level l
};

extern "C" orc_hb* orc_hb_create(uint64_t n_bits, int width, int all_set) {
    if (width < 2 || width > 64) return nullptr;
    orc_hb* h = new orc_hb;
    h->width = width;
    uint64_t n = n_bits;
    h->lv.emplace_back(n, all_set ? 1 : 0);
    while (n > (uint64_t)width) {
        uint64_t up = (n + width - 1) / width;
        h->lv.emplace_back(up, 0);
        n = up;
    }
    // Nested bits from their containers (container consistency).
    for (size_t l = 0; l + 1 < h->lv.size(); ++l)
        for (uint64_t i = 0; i < h->lv[l].size(); ++i)
            if (h->lv[l][i]) h->lv[l + 1][i / width] = 1;
    return h;
}

extern "C" void orc_hb_destroy(orc_hb* h) { delete h; }
extern "C" int orc_hb_levels(const orc_hb* h) { return (int)h->lv.size(); }
extern "C" uint64_t orc_hb_level_bits(const orc_hb* h, int l) { return h->lv[l].size(); }
extern "C" int orc_hb_get(const orc_hb* h, int l, uint64_t pos) { return h->lv[l][pos]; }

static bool container_empty(const orc_hb* h, size_t l, uint64_t cid) {
    const auto& v = h->lv[l];
    uint64_t lo = cid * h->width, hi = lo + h->width;
    if (hi > v.size()) hi = v.size();
    for (uint64_t i = lo; i < hi; ++i)
        if (v[i]) return false;
    return true;
}

static void push(int64_t* trace, int* n, size_t l, uint64_t pos) {
    if (trace) {
        trace[2 * *n] = (int64_t)l;
        trace[2 * *n + 1] = (int64_t)pos;
    }
    ++*n;
}

static int try_clear_at(orc_hb* h, size_t l, uint64_t pos, int64_t* trace, int* n) {
    if (!h->lv[l][pos]) return 0;
    h->lv[l][pos] = 0;
    push(trace, n, l, pos);
    uint64_t cid = pos / h->width;
    // This call cleared the last set bit of the container: its nested bit
    // must be cleared too (Alg. 2).
    if (l + 1 < h->lv.size() && container_empty(h, l, cid)) try_clear_at(h, l + 1, cid, trace, n);
    return 1;
}

static int try_set_at(orc_hb* h, size_t l, uint64_t pos, int64_t* trace, int* n) {
    if (h->lv[l][pos]) return 0;
    uint64_t cid = pos / h->width;
    bool was_empty = container_empty(h, l, cid);
    h->lv[l][pos] = 1;
    push(trace, n, l, pos);
    if (l + 1 < h->lv.size() && was_empty) try_set_at(h, l + 1, cid, trace, n);
    return 1;
}

extern "C" int orc_hb_try_clear(orc_hb* h, uint64_t pos, int64_t* trace, int* n_trace) {
    int n = 0;
    int r = try_clear_at(h, 0, pos, trace, &n);
    if (n_trace) *n_trace = n;
    return r;
}

extern "C" int orc_hb_try_set(orc_hb* h, uint64_t pos, int64_t* trace, int* n_trace) {
    int n = 0;
    int r = try_set_at(h, 0, pos, trace, &n);
    if (n_trace) *n_trace = n;
    return r;
}

extern "C" int64_t orc_hb_try_find_set(const orc_hb* h) {
    size_t top = h->lv.size() - 1;
    // Top level fits in one container.
    uint64_t lo = 0, hi = h->lv[top].size();
    for (size_t l = top + 1; l-- > 0;) {
        const auto& v = h->lv[l];
        if (hi > v.size()) hi = v.size();
        int64_t found = -1;
        for (uint64_t i = lo; i < hi; ++i)
            if (v[i]) { found = (int64_t)i; break; }
        if (found < 0) return -1;
        if (l == 0) return found;
        lo = (uint64_t)found * h->width;
        hi = lo + h->width;
    }
    return -1;
}

extern "C" int64_t orc_hb_clear_any(orc_hb* h) {
    int64_t i = orc_hb_try_find_set(h);
    if (i < 0) return -1;
    int n = 0;
    return try_clear_at(h, 0, (uint64_t)i, nullptr, &n) ? i : -1;
}

extern "C" int orc_hb_consistent(const orc_hb* h) {
    for (size_t l = 0; l + 1 < h->lv.size(); ++l)
        for (uint64_t c = 0; c < h->lv[l + 1].size(); ++c)
            if ((int)h->lv[l + 1][c] != (container_empty(h, l, c) ? 0 : 1)) return 0;
    return 1;
}

// ---------------------------------------------------------------------------
// Heap invariant checker (Section 2 "Block States", Fig. 2; Section 3
// container consistency). Reading of the block states used here: a block is
// either free or allocated[T] for exactly one T; an allocated[T] block holds
// objects of type T only and at least one of them; active[T] is set exactly
// for allocated[T] blocks with at least one free slot (active => allocated).
// At a quiescent point (no operation in flight) every bitmap is consistent.
// ---------------------------------------------------------------------------
// Bit i of a bitmap level whose 64-bit words each hold `width` bits.
static inline int bit_of(const uint64_t* w, uint64_t i, unsigned width) {
    return (int)((w[i / width] >> (i % width)) & 1u);
}

static int popc64(uint64_t x) {
    int c = 0;
    while (x) { x &= x - 1; ++c; }
    return c;
}

extern "C" uint32_t orc_check_heap(uint64_t M, int n_types, const uint32_t* capacity,
                                   const uint64_t* obj_free, const uint8_t* block_type,
                                   const uint64_t* free_bm, const uint64_t* alloc_bm,
                                   const uint64_t* active_bm, const uint64_t* words_per_level,
                                   int n_levels, int width, uint64_t* live_out) {
    uint32_t bad = 0;
    if (width != 16 && width != 32 && width != 64) return 32;
    const uint64_t W = (uint64_t)width;
    // Expected level structure for containers of `width` bits: level l + 1
    // has one bit per container of level l (Section 3).
    std::vector<uint64_t> bits_l, off_l;
    {
        uint64_t n = M, off = 0;
        bits_l.push_back(n);
        while (n > W) { n = (n + W - 1) / W; bits_l.push_back(n); }
        if ((int)bits_l.size() != n_levels) return 32;
        for (int l = 0; l < n_levels; ++l) {
            if (words_per_level[l] != (bits_l[l] + W - 1) / W) return 32;
            off_l.push_back(off);
            off += words_per_level[l];
        }
    }
    uint64_t total_words = off_l.back() + words_per_level[n_levels - 1];
    const uint64_t unused = W == 64 ? 0 : ~((1ull << W) - 1);  // word bits beyond the width

    auto check_bitmap = [&](const uint64_t* bm) {
        for (int l = 0; l < n_levels; ++l) {
            const uint64_t* w = bm + off_l[l];
            // no bit at or beyond the level's size, none beyond a word's width
            for (uint64_t i = bits_l[l]; i < words_per_level[l] * W; ++i)
                if (bit_of(w, i, width)) bad |= 16;
            for (uint64_t c = 0; c < words_per_level[l]; ++c)
                if (w[c] & unused) bad |= 16;
            if (l + 1 < n_levels) {
                const uint64_t* up = bm + off_l[l + 1];
                for (uint64_t c = 0; c < words_per_level[l]; ++c) {
                    int any = w[c] != 0;
                    if (any != bit_of(up, c, width)) bad |= 1;
                }
            }
        }
    };
    check_bitmap(free_bm);
    for (int t = 0; t < n_types; ++t) {
        check_bitmap(alloc_bm + (uint64_t)t * total_words);
        check_bitmap(active_bm + (uint64_t)t * total_words);
    }

    for (int t = 0; t < n_types; ++t) live_out[t] = 0;
    for (uint64_t b = 0; b < M; ++b) {
        int states = bit_of(free_bm, b, width);
        for (int t = 0; t < n_types; ++t) {
            const uint64_t* al = alloc_bm + (uint64_t)t * total_words;
            const uint64_t* ac = active_bm + (uint64_t)t * total_words;
            int a = bit_of(al, b, width), act = bit_of(ac, b, width);
            states += a;
            if (a) {
                uint64_t valid = capacity[t] >= 64 ? ~0ull : ((1ull << capacity[t]) - 1);
                uint64_t fr = obj_free[b];
                if (block_type[b] != (uint8_t)t) bad |= 4;
                if (fr & ~valid) bad |= 16;
                int live = (int)capacity[t] - popc64(fr & valid);
                if (live < 1) bad |= 4;
                live_out[t] += (uint64_t)(live > 0 ? live : 0);
                int want_active = (fr & valid) != 0;
                if (act != want_active) bad |= 8;
            } else if (act) {
                bad |= 8;
            }
        }
        if (states != 1) bad |= 2;
    }
    return bad;
}
