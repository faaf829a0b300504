// Oracle: n-body with merging collisions, FP64 (Fig. 6b/6d, "collisions" and
// "nbody: particle system"; Fig. 1 names an Euler time step). Test
// infrastructure only.
//
// The paper names the applications only. Rules fixed for both this oracle and
// the GPU path:
//   force:  a_i = G * sum_{j != i} m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2)
//   update: v_i += a_i dt, then x_i += v_i dt (semi-implicit Euler)
//   merge:  on the updated positions, the partner p(i) of body i is the body
//           with the lowest id j != i with |x_i - x_j| < r_merge (none if no
//           such body). Bodies i < j merge iff p(i) = j and p(j) = i: body i
//           takes m = m_i + m_j and the mass-weighted mean of position and
//           velocity (momentum is conserved), and body j is deleted. Bodies in
//           an unmatched chain wait for a later step.
// Objects: Body {id, x, y, z, vx, vy, vz, m}; trivial allocator (a vector and a
// live flag).
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

struct orc_nbody {
    orc_nbody_params p;
    int64_t step = 0;
    std::vector<double> x, y, z, vx, vy, vz, m;
    std::vector<uint8_t> live;
};

extern "C" orc_nbody* orc_nbody_create(const orc_nbody_params* p, const double* rows, int64_t n) {
    orc_nbody* b = new orc_nbody;
    b->p = *p;
    for (int64_t i = 0; i < n; ++i) {
        const double* r = rows + 7 * i;
        b->x.push_back(r[0]); b->y.push_back(r[1]); b->z.push_back(r[2]);
        b->vx.push_back(r[3]); b->vy.push_back(r[4]); b->vz.push_back(r[5]);
        b->m.push_back(r[6]);
        b->live.push_back(1);
    }
    return b;
}

extern "C" void orc_nbody_destroy(orc_nbody* b) { delete b; }

// Rows i of the force and partner loops are independent; they may be split
// across threads (orc_set_threads). Each row is computed the same way, in the
// same j order, whatever the thread count, so results do not depend on it.
static int g_threads = 1;

extern "C" void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

template <class F>
static void for_rows(int64_t n, F fn) {
    if (g_threads <= 1 || n < 256) {
        fn(0, n, 0);
        return;
    }
    std::vector<std::thread> th;
    const int64_t chunk = (n + g_threads - 1) / g_threads;
    for (int t = 0; t < g_threads; ++t) {
        const int64_t lo = t * chunk, hi = std::min<int64_t>(n, lo + chunk);
        if (lo < hi) th.emplace_back(fn, lo, hi, t);
    }
    for (auto& x : th) x.join();
}

extern "C" int64_t orc_nbody_step(orc_nbody* b, int n_steps, int64_t* merges_out, int64_t merges_cap,
                                  double margin, int64_t* marginal_out) {
    const auto& P = b->p;
    const int64_t n = (int64_t)b->x.size();
    int64_t n_merges = 0, n_marginal = 0;
    std::vector<double> ax(n), ay(n), az(n);
    std::vector<int64_t> partner(n);
    std::vector<int64_t> marg(g_threads > 1 ? g_threads : 1);
    for (int s = 0; s < n_steps; ++s) {
        // force
        for_rows(n, [&](int64_t lo, int64_t hi, int) {
            for (int64_t i = lo; i < hi; ++i) {
                if (!b->live[i]) continue;
                double sx = 0, sy = 0, sz = 0;
                for (int64_t j = 0; j < n; ++j) {
                    if (j == i || !b->live[j]) continue;
                    double dx = b->x[j] - b->x[i], dy = b->y[j] - b->y[i], dz = b->z[j] - b->z[i];
                    double r2 = dx * dx + dy * dy + dz * dz + P.eps * P.eps;
                    double w = b->m[j] / (r2 * std::sqrt(r2));
                    sx += w * dx; sy += w * dy; sz += w * dz;
                }
                ax[i] = P.G * sx; ay[i] = P.G * sy; az[i] = P.G * sz;
            }
        });
        // update
        for (int64_t i = 0; i < n; ++i) {
            if (!b->live[i]) continue;
            b->vx[i] += ax[i] * P.dt; b->vy[i] += ay[i] * P.dt; b->vz[i] += az[i] * P.dt;
            b->x[i] += b->vx[i] * P.dt; b->y[i] += b->vy[i] * P.dt; b->z[i] += b->vz[i] * P.dt;
        }
        // merge partners: lowest id within r_merge
        const double r2m = P.r_merge * P.r_merge;
        std::fill(marg.begin(), marg.end(), 0);
        for_rows(n, [&](int64_t lo, int64_t hi, int t) {
            for (int64_t i = lo; i < hi; ++i) {
                partner[i] = -1;
                if (!b->live[i]) continue;
                for (int64_t j = 0; j < n; ++j) {
                    if (j == i || !b->live[j]) continue;
                    double dx = b->x[j] - b->x[i], dy = b->y[j] - b->y[i], dz = b->z[j] - b->z[i];
                    double d2 = dx * dx + dy * dy + dz * dz;
                    if (margin > 0 && j > i && std::fabs(std::sqrt(d2) - P.r_merge) < margin) ++marg[t];
                    if (partner[i] < 0 && d2 < r2m) {
                        partner[i] = j;
                        if (margin <= 0) break;
                    }
                }
            }
        });
        for (int64_t m : marg) n_marginal += m;
        // merge mutual pairs; the lower id survives
        for (int64_t i = 0; i < n; ++i) {
            int64_t j = partner[i];
            if (j <= i || partner[j] != i) continue;
            double mi = b->m[i], mj = b->m[j], M = mi + mj;
            b->vx[i] = (mi * b->vx[i] + mj * b->vx[j]) / M;
            b->vy[i] = (mi * b->vy[i] + mj * b->vy[j]) / M;
            b->vz[i] = (mi * b->vz[i] + mj * b->vz[j]) / M;
            b->x[i] = (mi * b->x[i] + mj * b->x[j]) / M;
            b->y[i] = (mi * b->y[i] + mj * b->y[j]) / M;
            b->z[i] = (mi * b->z[i] + mj * b->z[j]) / M;
            b->m[i] = M;
            b->live[j] = 0;
            if (merges_out && n_merges < merges_cap) {
                merges_out[3 * n_merges + 0] = b->step;
                merges_out[3 * n_merges + 1] = i;
                merges_out[3 * n_merges + 2] = j;
            }
            ++n_merges;
        }
        b->step += 1;
    }
    if (marginal_out) *marginal_out = n_marginal;
    return n_merges;
}

extern "C" int64_t orc_nbody_count(const orc_nbody* b) {
    int64_t c = 0;
    for (auto u : b->live) c += u;
    return c;
}

extern "C" int64_t orc_nbody_dump(const orc_nbody* b, double* out, int64_t cap) {
    int64_t k = 0;
    for (size_t i = 0; i < b->x.size(); ++i) {
        if (!b->live[i]) continue;
        if (k >= cap) return -1;
        double* r = out + 8 * k;
        r[0] = (double)i;
        r[1] = b->x[i]; r[2] = b->y[i]; r[3] = b->z[i];
        r[4] = b->vx[i]; r[5] = b->vy[i]; r[6] = b->vz[i];
        r[7] = b->m[i];
        ++k;
    }
    return k;
}
