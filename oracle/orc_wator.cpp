// Oracle: wa-tor predator-prey as an SMMO program (Fig. 6h, "wator:
// agent-based simulation"; Dewdney's Wa-Tor). Test infrastructure only.
//
// The paper names the application only. The rules, fixed for both this oracle
// and the GPU path, on a W x H torus with von Neumann neighbours taken in the
// order N (y-1), E (x+1), S (y+1), W (x-1); cell index = y*W + x:
//   F1 do-all Fish:  timer += 1; candidates = empty neighbours in the grid as
//                    it is at the start of the step; if there are k > 0, pick
//                    candidate (r mod k) with r = rand(seed, 0, step, cell) and
//                    claim the target; the claim with the lowest mover cell
//                    index wins.
//   F2 do-all Fish:  a winner moves; if timer >= fish_breed it leaves a new
//                    Fish (timer 0) in the cell it left and resets timer to 0.
//   S0 do-all Shark: energy -= 1; at 0 the shark leaves the grid and is deleted.
//   S1 do-all Shark: timer += 1; candidates = neighbours holding a fish, or if
//                    there are none, empty neighbours (grid after F2 and S0);
//                    pick (r mod k) with r = rand(seed, 1, step, cell); claim,
//                    lowest mover cell index wins.
//   S2 do-all Shark: a winner moves; if the target held a fish, that Fish is
//                    deleted and energy += shark_gain; if timer >= shark_breed
//                    it leaves a new Shark (timer 0, energy shark_energy0) and
//                    resets timer to 0.
// A do-all visits the objects that are live when it starts. Objects: Fish
// {x, y, timer}, Shark {x, y, timer, energy}; trivial allocator (vector +
// free list per type).
#include "oracle.h"

#include <algorithm>
#include <array>
#include <climits>
#include <vector>

namespace {
enum : uint8_t { EMPTY = 0, FISH = 1, SHARK = 2 };

template <int K>
struct Pool {
    std::vector<std::array<int32_t, K>> obj;
    std::vector<uint8_t> used;
    std::vector<int64_t> free_list;
    int64_t add(const std::array<int32_t, K>& v) {
        if (!free_list.empty()) {
            int64_t i = free_list.back();
            free_list.pop_back();
            obj[i] = v;
            used[i] = 1;
            return i;
        }
        obj.push_back(v);
        used.push_back(1);
        return (int64_t)obj.size() - 1;
    }
    void remove(int64_t i) {
        used[i] = 0;
        free_list.push_back(i);
    }
    std::vector<int64_t> live() const {
        std::vector<int64_t> v;
        for (size_t i = 0; i < used.size(); ++i)
            if (used[i]) v.push_back((int64_t)i);
        return v;
    }
};
}  // namespace

struct orc_wator {
    orc_wator_params p;
    int64_t step = 0;
    std::vector<uint8_t> kind;      // per cell
    std::vector<int64_t> occupant;  // per cell: object index in its pool
    std::vector<int64_t> claim;     // per cell: lowest claiming mover cell, LLONG_MAX = none
    Pool<3> fish;                   // x, y, timer
    Pool<4> shark;                  // x, y, timer, energy

    int64_t cell_of(int32_t x, int32_t y) const { return (int64_t)y * p.W + x; }
    void neighbours(int64_t c, int64_t out[4]) const {
        int32_t x = (int32_t)(c % p.W), y = (int32_t)(c / p.W);
        out[0] = cell_of(x, (y - 1 + p.H) % p.H);  // N
        out[1] = cell_of((x + 1) % p.W, y);        // E
        out[2] = cell_of(x, (y + 1) % p.H);        // S
        out[3] = cell_of((x - 1 + p.W) % p.W, y);  // W
    }
};

extern "C" orc_wator* orc_wator_create(const orc_wator_params* p, const uint8_t* kind0) {
    orc_wator* w = new orc_wator;
    w->p = *p;
    int64_t n = (int64_t)p->W * p->H;
    w->kind.assign(kind0, kind0 + n);
    w->occupant.assign(n, -1);
    w->claim.assign(n, LLONG_MAX);
    for (int64_t c = 0; c < n; ++c) {
        int32_t x = (int32_t)(c % p->W), y = (int32_t)(c / p->W);
        if (kind0[c] == FISH) w->occupant[c] = w->fish.add({x, y, 0});
        else if (kind0[c] == SHARK) w->occupant[c] = w->shark.add({x, y, 0, p->shark_energy0});
        else w->kind[c] = EMPTY;
    }
    return w;
}

extern "C" void orc_wator_destroy(orc_wator* w) { delete w; }

extern "C" void orc_wator_step(orc_wator* w, int n_steps, int64_t* events_out) {
    const auto& P = w->p;
    for (int s = 0; s < n_steps; ++s) {
        const uint64_t t = (uint64_t)w->step;
        int64_t fish_births = 0, eaten = 0, shark_births = 0, starved = 0, fish_moves = 0, shark_moves = 0;

        // ---- F1: fish choose a target among empty neighbours and claim it.
        std::vector<int64_t> fl = w->fish.live();
        std::vector<int64_t> intent(fl.size(), -1);
        for (size_t k = 0; k < fl.size(); ++k) {
            auto& f = w->fish.obj[fl[k]];
            f[2] += 1;
            int64_t c = w->cell_of(f[0], f[1]), nb[4], cand[4];
            w->neighbours(c, nb);
            int nc = 0;
            for (int d = 0; d < 4; ++d)
                if (w->kind[nb[d]] == EMPTY) cand[nc++] = nb[d];
            if (nc == 0) continue;
            int64_t tgt = cand[orc_rand(P.seed, 0, t, (uint64_t)c) % (uint64_t)nc];
            intent[k] = tgt;
            w->claim[tgt] = std::min(w->claim[tgt], c);
        }
        // ---- F2: winners move, and breed when old enough.
        for (size_t k = 0; k < fl.size(); ++k) {
            int64_t tgt = intent[k];
            if (tgt < 0) continue;
            auto& f = w->fish.obj[fl[k]];
            int64_t c = w->cell_of(f[0], f[1]);
            if (w->claim[tgt] != c) continue;
            ++fish_moves;
            w->kind[tgt] = FISH;
            w->occupant[tgt] = fl[k];
            f[0] = (int32_t)(tgt % P.W);
            f[1] = (int32_t)(tgt / P.W);
            if (f[2] >= P.fish_breed) {
                f[2] = 0;
                int64_t nf = w->fish.add({(int32_t)(c % P.W), (int32_t)(c / P.W), 0});
                w->kind[c] = FISH;
                w->occupant[c] = nf;
                ++fish_births;
            } else {
                w->kind[c] = EMPTY;
                w->occupant[c] = -1;
            }
        }
        for (int64_t tgt : intent)
            if (tgt >= 0) w->claim[tgt] = LLONG_MAX;

        // ---- S0: starvation.
        std::vector<int64_t> sl = w->shark.live();
        for (int64_t i : sl) {
            auto& sh = w->shark.obj[i];
            sh[3] -= 1;
            if (sh[3] == 0) {
                int64_t c = w->cell_of(sh[0], sh[1]);
                w->kind[c] = EMPTY;
                w->occupant[c] = -1;
                w->shark.remove(i);
                ++starved;
            }
        }
        // ---- S1: sharks prefer a neighbouring fish, else an empty cell.
        sl = w->shark.live();
        std::vector<int64_t> sint(sl.size(), -1);
        for (size_t k = 0; k < sl.size(); ++k) {
            auto& sh = w->shark.obj[sl[k]];
            sh[2] += 1;
            int64_t c = w->cell_of(sh[0], sh[1]), nb[4], cand[4];
            w->neighbours(c, nb);
            int nc = 0;
            for (int d = 0; d < 4; ++d)
                if (w->kind[nb[d]] == FISH) cand[nc++] = nb[d];
            if (nc == 0)
                for (int d = 0; d < 4; ++d)
                    if (w->kind[nb[d]] == EMPTY) cand[nc++] = nb[d];
            if (nc == 0) continue;
            int64_t tgt = cand[orc_rand(P.seed, 1, t, (uint64_t)c) % (uint64_t)nc];
            sint[k] = tgt;
            w->claim[tgt] = std::min(w->claim[tgt], c);
        }
        // ---- S2: winners move, eat, and breed.
        for (size_t k = 0; k < sl.size(); ++k) {
            int64_t tgt = sint[k];
            if (tgt < 0) continue;
            auto& sh = w->shark.obj[sl[k]];
            int64_t c = w->cell_of(sh[0], sh[1]);
            if (w->claim[tgt] != c) continue;
            ++shark_moves;
            if (w->kind[tgt] == FISH) {
                w->fish.remove(w->occupant[tgt]);
                sh[3] += P.shark_gain;
                ++eaten;
            }
            w->kind[tgt] = SHARK;
            w->occupant[tgt] = sl[k];
            sh[0] = (int32_t)(tgt % P.W);
            sh[1] = (int32_t)(tgt / P.W);
            if (sh[2] >= P.shark_breed) {
                sh[2] = 0;
                int64_t ns = w->shark.add({(int32_t)(c % P.W), (int32_t)(c / P.W), 0, P.shark_energy0});
                w->kind[c] = SHARK;
                w->occupant[c] = ns;
                ++shark_births;
            } else {
                w->kind[c] = EMPTY;
                w->occupant[c] = -1;
            }
        }
        for (int64_t tgt : sint)
            if (tgt >= 0) w->claim[tgt] = LLONG_MAX;

        if (events_out) {
            int64_t* e = events_out + 6 * s;
            e[0] = fish_births;
            e[1] = eaten;
            e[2] = shark_births;
            e[3] = starved;
            e[4] = fish_moves;
            e[5] = shark_moves;
        }
        w->step += 1;
    }
}

extern "C" void orc_wator_counts(const orc_wator* w, int64_t* n_fish, int64_t* n_shark) {
    int64_t a = 0, b = 0;
    for (auto u : w->fish.used) a += u;
    for (auto u : w->shark.used) b += u;
    *n_fish = a;
    *n_shark = b;
}

extern "C" void orc_wator_hash(const orc_wator* w, uint64_t* fish_hash, uint64_t* shark_hash) {
    // Type ids: Fish = 0, Shark = 1.
    uint64_t hf = 0, hs = 0;
    for (size_t i = 0; i < w->fish.obj.size(); ++i) {
        if (!w->fish.used[i]) continue;
        const auto& f = w->fish.obj[i];
        uint32_t v[3] = {(uint32_t)f[0], (uint32_t)f[1], (uint32_t)f[2]};
        hf += orc_obj_hash(0, v, 3);
    }
    for (size_t i = 0; i < w->shark.obj.size(); ++i) {
        if (!w->shark.used[i]) continue;
        const auto& s = w->shark.obj[i];
        uint32_t v[4] = {(uint32_t)s[0], (uint32_t)s[1], (uint32_t)s[2], (uint32_t)s[3]};
        hs += orc_obj_hash(1, v, 4);
    }
    *fish_hash = hf;
    *shark_hash = hs;
}

extern "C" int orc_wator_dump(const orc_wator* w, int32_t* fish_out, int64_t fish_cap,
                              int32_t* shark_out, int64_t shark_cap) {
    std::vector<std::array<int32_t, 3>> f;
    std::vector<std::array<int32_t, 4>> s;
    for (size_t i = 0; i < w->fish.obj.size(); ++i)
        if (w->fish.used[i]) f.push_back(w->fish.obj[i]);
    for (size_t i = 0; i < w->shark.obj.size(); ++i)
        if (w->shark.used[i]) s.push_back(w->shark.obj[i]);
    if ((int64_t)f.size() > fish_cap || (int64_t)s.size() > shark_cap) return -1;
    std::sort(f.begin(), f.end());
    std::sort(s.begin(), s.end());
    for (size_t i = 0; i < f.size(); ++i)
        for (int k = 0; k < 3; ++k) fish_out[3 * i + k] = f[i][k];
    for (size_t i = 0; i < s.size(); ++i)
        for (int k = 0; k < 4; ++k) shark_out[4 * i + k] = s[i][k];
    return 0;
}

extern "C" void orc_wator_grid(const orc_wator* w, uint8_t* kind_out) {
    std::copy(w->kind.begin(), w->kind.end(), kind_out);
}
