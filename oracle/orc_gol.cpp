// Oracle: game of life as an SMMO program (Fig. 6c, "game-of-life: cellular
// automaton"). Test infrastructure only.
//
// The paper names the application only. The rules used (and stated the same
// way for the GPU path) are Conway's B3/S23 on a W x H torus with the Moore
// neighbourhood, written as three parallel do-alls per generation (Section
// 1.1: parallelism is a method run on all objects of a type; objects may be
// created and deleted inside a do-all):
//   (i)   do-all Cell:  count = number of alive cells among the 8 neighbours
//   (ii)  do-all Alive: if its cell's count is not 2 or 3, the cell dies and
//                       the Alive object deletes itself
//   (iii) do-all Cell:  if the cell is dead and count == 3 it becomes alive
//                       and a new Alive object is created for it
// Types: Cell {alive, count, idx} (idx = y*W + x, the cell's own position, so
// a Cell can find its neighbours) and Alive {x, y}.
// Storage is a trivial allocator: a vector per type plus a free list.
#include "oracle.h"

#include <algorithm>
#include <array>
#include <vector>

struct orc_gol {
    int W, H;
    std::vector<std::array<int32_t, 3>> cell;  // (alive, count, idx), cell i at index i
    std::vector<std::array<int32_t, 2>> alive; // Alive objects (x, y)
    std::vector<uint8_t> alive_used;
    std::vector<int64_t> free_list;

    int64_t new_alive(int32_t x, int32_t y) {
        int64_t i;
        if (!free_list.empty()) {
            i = free_list.back();
            free_list.pop_back();
            alive[i] = {x, y};
            alive_used[i] = 1;
        } else {
            i = (int64_t)alive.size();
            alive.push_back({x, y});
            alive_used.push_back(1);
        }
        return i;
    }
    void delete_alive(int64_t i) {
        alive_used[i] = 0;
        free_list.push_back(i);
    }
};

extern "C" orc_gol* orc_gol_create(int W, int H, const uint8_t* alive0) {
    orc_gol* g = new orc_gol;
    g->W = W;
    g->H = H;
    g->cell.resize((size_t)W * H);
    for (int i = 0; i < W * H; ++i) {
        g->cell[i] = {alive0[i] ? 1 : 0, 0, i};
        if (alive0[i]) g->new_alive(i % W, i / W);
    }
    return g;
}

extern "C" void orc_gol_destroy(orc_gol* g) { delete g; }

extern "C" void orc_gol_step(orc_gol* g, int n_gen) {
    const int W = g->W, H = g->H;
    for (int gen = 0; gen < n_gen; ++gen) {
        // (i) do-all Cell: neighbour count
        for (auto& c : g->cell) {
            int x = c[2] % W, y = c[2] / W, n = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (dx == 0 && dy == 0) continue;
                    int nx = (x + dx + W) % W, ny = (y + dy + H) % H;
                    n += g->cell[(size_t)ny * W + nx][0];
                }
            c[1] = n;
        }
        // (ii) do-all Alive: death by under- or over-population
        for (int64_t i = 0; i < (int64_t)g->alive.size(); ++i) {
            if (!g->alive_used[i]) continue;
            auto& c = g->cell[(size_t)g->alive[i][1] * W + g->alive[i][0]];
            if (c[1] != 2 && c[1] != 3) {
                c[0] = 0;
                g->delete_alive(i);
            }
        }
        // (iii) do-all Cell: birth
        for (auto& c : g->cell) {
            if (!c[0] && c[1] == 3) {
                c[0] = 1;
                g->new_alive(c[2] % W, c[2] / W);
            }
        }
    }
}

extern "C" int64_t orc_gol_alive_count(const orc_gol* g) {
    int64_t n = 0;
    for (auto u : g->alive_used) n += u;
    return n;
}

extern "C" void orc_gol_hash(const orc_gol* g, uint64_t* cell_hash, uint64_t* alive_hash) {
    // Type ids: Cell = 0, Alive = 1.
    uint64_t hc = 0, ha = 0;
    for (auto& c : g->cell) {
        uint32_t w[3] = {(uint32_t)c[0], (uint32_t)c[1], (uint32_t)c[2]};
        hc += orc_obj_hash(0, w, 3);
    }
    for (size_t i = 0; i < g->alive.size(); ++i) {
        if (!g->alive_used[i]) continue;
        uint32_t w[2] = {(uint32_t)g->alive[i][0], (uint32_t)g->alive[i][1]};
        ha += orc_obj_hash(1, w, 2);
    }
    *cell_hash = hc;
    *alive_hash = ha;
}

extern "C" int64_t orc_gol_dump(const orc_gol* g, int32_t* cells_out, int32_t* alive_out, int64_t cap) {
    for (size_t i = 0; i < g->cell.size(); ++i)
        for (int k = 0; k < 3; ++k) cells_out[3 * i + k] = g->cell[i][k];
    std::vector<std::array<int32_t, 2>> a;
    for (size_t i = 0; i < g->alive.size(); ++i)
        if (g->alive_used[i]) a.push_back(g->alive[i]);
    std::sort(a.begin(), a.end());
    if ((int64_t)a.size() > cap) return -1;
    for (size_t i = 0; i < a.size(); ++i) {
        alive_out[2 * i] = a[i][0];
        alive_out[2 * i + 1] = a[i][1];
    }
    return (int64_t)a.size();
}
