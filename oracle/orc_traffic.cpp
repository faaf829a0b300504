// Oracle: traffic as an SMMO program (Fig. 6g, "traffic": the
// Nagel-Schreckenberg model). Test infrastructure only.
//
// The paper names the application and the model only. The rules, fixed for
// both this oracle and the GPU path, are the published Nagel-Schreckenberg
// cellular automaton (Nagel and Schreckenberg, J. Phys. I France 2, 1992) on
// R independent single-lane roads of L cells, with parallel update. Objects:
// Car {road, x, v}; on open roads one Source {road, entered, blocked} per
// road. Per step t (counting from 0), with every read of occupancy taken
// from the positions at the start of the step:
//   do-all Car:    v1 = min(v + 1, vmax)                        (acceleration)
//                  g  = free cells ahead before the next car, looking at
//                       most v1 cells ahead; on an open road cells past the
//                       end are free, on a periodic road the road wraps
//                  v2 = min(v1, g)                               (slowing down)
//                  v3 = max(v2 - 1, 0) if rand(seed, 5, t, road * L + x)
//                       draws below p, else v2                   (randomisation)
//                  x' = x + v3                                   (motion); on
//                       an open road a car with x' >= L leaves and is
//                       deleted; on a periodic road x' wraps
//   do-all Source: (open roads) if cell 0 of its road is free after the car
//                  do-all and rand(seed, 6, t, road) draws below alpha, a
//                  new Car(road, 0, v_entry) enters and `entered` grows by 1;
//                  if cell 0 is occupied, `blocked` grows by 1.
// "Draws below p": (r >> 32) < p_thr, with p_thr = floor(p * 2^32) (2^32 for
// p = 1). Cars move within the free cells ahead of them, so no two cars
// target one cell and the result does not depend on the order of the do-all.
// A do-all visits the objects live when it starts (new cars wait a step).
#include "oracle.h"

#include <algorithm>
#include <array>
#include <vector>

struct orc_traffic {
    orc_traffic_params p;
    int64_t step = 0;
    std::vector<std::array<int32_t, 3>> cars;     // road, x, v (live cars; order irrelevant)
    std::vector<std::array<int32_t, 3>> sources;  // road, entered, blocked
    std::vector<uint8_t> occ;                     // [R * L] occupancy at the start of the step
};

extern "C" orc_traffic* orc_traffic_create(const orc_traffic_params* p, const int8_t* v0) {
    if (!p || !v0 || p->R < 1 || p->L <= p->vmax || p->vmax < 1 || p->v_entry < 0 || p->v_entry > p->vmax)
        return nullptr;
    orc_traffic* t = new orc_traffic;
    t->p = *p;
    t->occ.assign((size_t)p->R * p->L, 0);
    for (int32_t r = 0; r < p->R; ++r)
        for (int32_t x = 0; x < p->L; ++x) {
            const int8_t v = v0[(size_t)r * p->L + x];
            if (v < 0) continue;
            t->cars.push_back({r, x, std::min<int32_t>(v, p->vmax)});
            t->occ[(size_t)r * p->L + x] = 1;
        }
    if (!p->periodic)
        for (int32_t r = 0; r < p->R; ++r) t->sources.push_back({r, 0, 0});
    return t;
}

extern "C" void orc_traffic_destroy(orc_traffic* t) { delete t; }

extern "C" void orc_traffic_step(orc_traffic* t, int n_steps, int64_t* events_out) {
    const orc_traffic_params& p = t->p;
    const int64_t L = p.L;
    for (int s = 0; s < n_steps; ++s) {
        int64_t entries = 0, exits = 0, moving = 0, vsum = 0;
        std::vector<uint8_t> next(t->occ.size(), 0);
        std::vector<std::array<int32_t, 3>> kept;
        kept.reserve(t->cars.size());
        // do-all Car (reads t->occ, the start-of-step positions)
        for (const auto& c : t->cars) {
            const int32_t road = c[0], x = c[1], v = c[2];
            const int32_t v1 = std::min(v + 1, p.vmax);
            int32_t g = 0;
            while (g < v1) {
                int64_t ahead = x + g + 1;
                if (ahead >= L) {
                    if (!p.periodic) {  // past the end of an open road: free
                        ++g;
                        continue;
                    }
                    ahead -= L;
                }
                if (t->occ[(size_t)road * L + ahead]) break;
                ++g;
            }
            int32_t v3 = std::min(v1, g);
            const uint64_t r = orc_rand(p.seed, 5, (uint64_t)t->step, (uint64_t)road * L + x);
            if ((r >> 32) < p.p_thr) v3 = std::max(v3 - 1, 0);
            vsum += v3;
            if (v3 > 0) ++moving;
            int64_t nx = (int64_t)x + v3;
            if (nx >= L) {
                if (!p.periodic) {
                    ++exits;  // leaves the road: delete
                    continue;
                }
                nx -= L;
            }
            next[(size_t)road * L + nx] = 1;
            kept.push_back({road, (int32_t)nx, v3});
        }
        // do-all Source (open roads; sees the positions after the car do-all)
        for (auto& src : t->sources) {
            const int32_t road = src[0];
            if (next[(size_t)road * L]) {
                ++src[2];
                continue;
            }
            const uint64_t r = orc_rand(p.seed, 6, (uint64_t)t->step, (uint64_t)road);
            if ((r >> 32) < p.a_thr) {
                kept.push_back({road, 0, p.v_entry});
                next[(size_t)road * L] = 1;
                ++src[1];
                ++entries;
            }
        }
        t->cars.swap(kept);
        t->occ.swap(next);
        ++t->step;
        if (events_out) {
            events_out[4 * s + 0] = entries;
            events_out[4 * s + 1] = exits;
            events_out[4 * s + 2] = moving;
            events_out[4 * s + 3] = vsum;
        }
    }
}

extern "C" int64_t orc_traffic_count(const orc_traffic* t) { return (int64_t)t->cars.size(); }

extern "C" void orc_traffic_hash(const orc_traffic* t, uint64_t* car_hash, uint64_t* source_hash) {
    uint64_t hc = 0, hs = 0;
    for (const auto& c : t->cars) {
        const uint32_t w[3] = {(uint32_t)c[0], (uint32_t)c[1], (uint32_t)c[2]};
        hc += orc_obj_hash(0, w, 3);
    }
    for (const auto& s : t->sources) {
        const uint32_t w[3] = {(uint32_t)s[0], (uint32_t)s[1], (uint32_t)s[2]};
        hs += orc_obj_hash(1, w, 3);
    }
    if (car_hash) *car_hash = hc;
    if (source_hash) *source_hash = hs;
}

extern "C" int64_t orc_traffic_dump(const orc_traffic* t, int32_t* cars_out, int64_t cap, int32_t* sources_out) {
    std::vector<std::array<int32_t, 3>> c = t->cars;
    std::sort(c.begin(), c.end());
    if ((int64_t)c.size() > cap) return -1;
    for (size_t i = 0; i < c.size(); ++i)
        for (int k = 0; k < 3; ++k) cars_out[3 * i + k] = c[i][k];
    if (sources_out)
        for (size_t i = 0; i < t->sources.size(); ++i)
            for (int k = 0; k < 3; ++k) sources_out[3 * i + k] = t->sources[i][k];
    return (int64_t)c.size();
}
