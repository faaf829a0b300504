// Oracle: sugarscape as an SMMO program (Fig. 6f, "sugarscape: agent-based
// simulation"; Epstein and Axtell, Growing Artificial Societies, 1996,
// chapter II). Test infrastructure only.
//
// The paper names the application only. The rules, fixed for both this
// oracle and the GPU path, on a W x H torus (cell index = y * W + x):
//   landscape: cell capacity cap in {0..4}; sugar starts at cap and, at the
//     end of every step, grows back by alpha up to cap (rule G_alpha).
//   Agent {x, y, sugar, metabolism, vision, age, max_age, dead}.
//   step t:
//   A1 do-all Agent (movement rule M, choice): candidates are the agent's own
//      cell (distance 0) and the cells up to `vision` away in the directions
//      N (y-1), E (x+1), S (y+1), W (x-1) that no agent occupies at the start
//      of the step. The target is the candidate with the most sugar, among
//      those the nearest, among those (same distance, order N, E, S, W) the
//      one at index (r >> 32) mod k, r = rand(seed, 12, t, own cell). A target
//      other than its own cell is claimed; the lowest claiming cell wins.
//   A2 do-all Agent (movement and harvest): a winner moves; every agent then
//      collects all the sugar of its cell (which drops to 0), pays its
//      metabolism, and ages by 1; it dies (dead = 1, still on its cell) if its
//      sugar is below 0 or its age has reached max_age.
//   A3 do-all Agent (replacement rule R, choice): a dead agent draws a cell
//      c = (rand(seed, 13, t, own cell) >> 32) mod (W * H); if no agent (dead
//      or alive) occupies c, it claims c; the lowest claiming cell wins.
//   A4 do-all Agent (replacement): a dead agent is deleted and a new agent
//      (age 0) created at c if it won c, else in the cell it leaves. The new
//      agent's sugar, metabolism, vision and max_age are lo + (r >> 32) mod
//      (hi - lo + 1) with r = rand(seed, 8 + k, t, its cell) for k = 0..3.
//   then sugar grows back (G_alpha).
// A do-all visits the agents live at its start, so the population is
// constant.
#include "oracle.h"

#include <algorithm>
#include <array>
#include <climits>
#include <vector>

namespace {
enum { AX, AY, SUGAR, METAB, VISION, AGE, MAXAGE, DEAD, NF };
using Agent = std::array<int32_t, NF>;
}  // namespace

struct orc_sugarscape {
    orc_sugarscape_params p;
    int64_t step = 0;
    std::vector<uint8_t> cap;
    std::vector<int32_t> sugar;
    std::vector<uint8_t> occ;
    std::vector<Agent> agents;

    int64_t cell(int32_t x, int32_t y) const { return (int64_t)y * p.W + x; }
    int32_t draw(uint64_t stream, int64_t c, int32_t lo, int32_t hi) const {
        const uint64_t r = orc_rand(p.seed, stream, (uint64_t)step, (uint64_t)c) >> 32;
        return lo + (int32_t)(r % (uint64_t)(hi - lo + 1));
    }
    Agent newborn(int64_t c) const {
        Agent a{};
        a[AX] = (int32_t)(c % p.W);
        a[AY] = (int32_t)(c / p.W);
        a[SUGAR] = draw(8, c, p.endow_lo, p.endow_hi);
        a[METAB] = draw(9, c, p.metab_lo, p.metab_hi);
        a[VISION] = draw(10, c, p.vision_lo, p.vision_hi);
        a[AGE] = 0;
        a[MAXAGE] = draw(11, c, p.age_lo, p.age_hi);
        a[DEAD] = 0;
        return a;
    }
};

extern "C" orc_sugarscape* orc_sugarscape_create(const orc_sugarscape_params* p, const uint8_t* cap,
                                                 const int32_t* agents0, int64_t n_agents) {
    if (!p || !cap || (n_agents && !agents0) || p->alpha < 1 || p->vision_lo < 1 || p->vision_hi < p->vision_lo ||
        p->W < 2 * p->vision_hi + 1 || p->H < 2 * p->vision_hi + 1 || p->metab_hi < p->metab_lo ||
        p->endow_hi < p->endow_lo || p->age_lo < 1 || p->age_hi < p->age_lo)
        return nullptr;
    orc_sugarscape* s = new orc_sugarscape;
    s->p = *p;
    const int64_t n = (int64_t)p->W * p->H;
    s->cap.assign(cap, cap + n);
    s->sugar.resize(n);
    for (int64_t c = 0; c < n; ++c) s->sugar[c] = cap[c];
    s->occ.assign(n, 0);
    for (int64_t i = 0; i < n_agents; ++i) {
        Agent a{};
        for (int k = 0; k < 7; ++k) a[k] = agents0[7 * i + k];
        a[DEAD] = 0;
        const int64_t c = s->cell(a[AX], a[AY]);
        if (s->occ[c]) {
            delete s;
            return nullptr;
        }
        s->occ[c] = 1;
        s->agents.push_back(a);
    }
    return s;
}

extern "C" void orc_sugarscape_destroy(orc_sugarscape* s) { delete s; }

extern "C" void orc_sugarscape_step(orc_sugarscape* s, int n_steps, int64_t* events_out) {
    const orc_sugarscape_params& p = s->p;
    const int64_t n = (int64_t)p.W * p.H;
    static const int DX[4] = {0, 1, 0, -1}, DY[4] = {-1, 0, 1, 0};  // N, E, S, W
    for (int st = 0; st < n_steps; ++st) {
        int64_t moves = 0, starved = 0, aged = 0, moved_away = 0, harvest = 0;
        std::vector<int64_t> claim(n, LLONG_MAX);
        std::vector<int64_t> target(s->agents.size());
        // A1
        for (size_t i = 0; i < s->agents.size(); ++i) {
            const Agent& a = s->agents[i];
            const int64_t own = s->cell(a[AX], a[AY]);
            int32_t best = s->sugar[own], best_d = 0;
            std::vector<int64_t> cand{own};
            for (int d = 1; d <= a[VISION]; ++d)
                for (int k = 0; k < 4; ++k) {
                    const int32_t x = ((a[AX] + DX[k] * d) % p.W + p.W) % p.W;
                    const int32_t y = ((a[AY] + DY[k] * d) % p.H + p.H) % p.H;
                    const int64_t c = s->cell(x, y);
                    if (s->occ[c]) continue;
                    const int32_t v = s->sugar[c];
                    if (v > best) {  // more sugar wins; equal sugar: the nearer (earlier) stays
                        best = v;
                        best_d = d;
                        cand.assign(1, c);
                    } else if (v == best && d == best_d) {
                        cand.push_back(c);
                    }
                }
            int64_t t = cand[0];
            if (cand.size() > 1) {
                const uint64_t r = orc_rand(p.seed, 12, (uint64_t)s->step, (uint64_t)own) >> 32;
                t = cand[r % cand.size()];
            }
            target[i] = t;
            if (t != own) claim[t] = std::min(claim[t], own);
        }
        // A2
        for (size_t i = 0; i < s->agents.size(); ++i) {
            Agent& a = s->agents[i];
            const int64_t own = s->cell(a[AX], a[AY]);
            int64_t c = own;
            if (target[i] != own && claim[target[i]] == own) {
                c = target[i];
                s->occ[own] = 0;
                s->occ[c] = 1;
                a[AX] = (int32_t)(c % p.W);
                a[AY] = (int32_t)(c / p.W);
                ++moves;
            }
            a[SUGAR] += s->sugar[c];
            harvest += s->sugar[c];
            s->sugar[c] = 0;
            a[SUGAR] -= a[METAB];
            a[AGE] += 1;
            if (a[SUGAR] < 0) {
                a[DEAD] = 1;
                ++starved;
            } else if (a[AGE] >= a[MAXAGE]) {
                a[DEAD] = 1;
                ++aged;
            }
        }
        // A3
        std::vector<int64_t> claim2(n, LLONG_MAX);
        for (const Agent& a : s->agents) {
            if (!a[DEAD]) continue;
            const int64_t own = s->cell(a[AX], a[AY]);
            const int64_t c = (int64_t)((orc_rand(p.seed, 13, (uint64_t)s->step, (uint64_t)own) >> 32) % (uint64_t)n);
            if (!s->occ[c]) claim2[c] = std::min(claim2[c], own);
        }
        // A4
        std::vector<Agent> born;
        std::vector<Agent> kept;
        for (const Agent& a : s->agents) {
            if (!a[DEAD]) {
                kept.push_back(a);
                continue;
            }
            const int64_t own = s->cell(a[AX], a[AY]);
            const int64_t c = (int64_t)((orc_rand(p.seed, 13, (uint64_t)s->step, (uint64_t)own) >> 32) % (uint64_t)n);
            int64_t at = own;
            if (claim2[c] == own) {
                at = c;
                s->occ[own] = 0;
                s->occ[c] = 1;
                ++moved_away;
            }
            born.push_back(s->newborn(at));
        }
        kept.insert(kept.end(), born.begin(), born.end());
        s->agents.swap(kept);
        // growback
        for (int64_t c = 0; c < n; ++c) s->sugar[c] = std::min<int32_t>(s->sugar[c] + p.alpha, s->cap[c]);
        ++s->step;
        if (events_out) {
            events_out[5 * st + 0] = moves;
            events_out[5 * st + 1] = starved;
            events_out[5 * st + 2] = aged;
            events_out[5 * st + 3] = moved_away;
            events_out[5 * st + 4] = harvest;
        }
    }
}

extern "C" int64_t orc_sugarscape_count(const orc_sugarscape* s) { return (int64_t)s->agents.size(); }

extern "C" uint64_t orc_sugarscape_hash(const orc_sugarscape* s) {
    uint64_t h = 0;
    for (const Agent& a : s->agents) {
        uint32_t w[NF];
        for (int k = 0; k < NF; ++k) w[k] = (uint32_t)a[k];
        h += orc_obj_hash(0, w, NF);
    }
    return h;
}

extern "C" int64_t orc_sugarscape_dump(const orc_sugarscape* s, int32_t* agents_out, int64_t cap,
                                       int32_t* sugar_out) {
    std::vector<Agent> a = s->agents;
    std::sort(a.begin(), a.end());
    if ((int64_t)a.size() > cap) return -1;
    for (size_t i = 0; i < a.size(); ++i)
        for (int k = 0; k < NF; ++k) agents_out[NF * i + k] = a[i][k];
    if (sugar_out) std::copy(s->sugar.begin(), s->sugar.end(), sugar_out);
    return (int64_t)a.size();
}
