// The paper's CPU uniform-grid method (Hesam et al., Sec. IV-A), as a timing
// baseline for the benchmark: every step rebuilds the grid (box edge = the
// largest contact distance; each box keeps its last agent, each agent the one
// added before it), sums Eq. 1 over the 27 boxes around every agent, and
// applies the Sec. III displacement (adherence test, explicit integration with
// m = rho (pi/6) d^3, cap of the displacement length).  float64 throughout,
// OpenMP over agents; agent state as structure of arrays.  Not part of the
// library and not the test oracle.
#include <omp.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <vector>

namespace {

struct Params {
    float k, gamma, adherence, dt, density, max_disp, contact_margin;
};

struct Grid {
    double origin[3], edge;
    int64_t dims[3];
    std::vector<int64_t> head;
    std::vector<int64_t> next;
};

void build_grid(const std::vector<double> *pos, const std::vector<double> &diam, double margin,
                Grid &g) {
    const int64_t n = (int64_t)diam.size();
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double dmax = 0.0;
#pragma omp parallel for reduction(min : lo[:3]) reduction(max : hi[:3]) reduction(max : dmax)
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], pos[a][i]);
            hi[a] = std::max(hi[a], pos[a][i]);
        }
        dmax = std::max(dmax, diam[i]);
    }
    // a contact pair is closer than the largest contact distance S; an edge a
    // hair above S keeps such pairs in adjacent boxes despite rounding
    g.edge = (dmax + 2.0 * margin) * (1.0 + 1e-12);
    int64_t nboxes = 1;
    for (int a = 0; a < 3; ++a) {
        g.origin[a] = lo[a] - g.edge;   // one empty layer of boxes all round
        g.dims[a] = (int64_t)std::floor((hi[a] - g.origin[a]) / g.edge) + 2;
        nboxes *= g.dims[a];
    }
    g.head.assign((size_t)nboxes, -1);
    g.next.resize((size_t)n);
#pragma omp parallel for
    for (int64_t i = 0; i < n; ++i) {
        int64_t b[3];
        for (int a = 0; a < 3; ++a)
            b[a] = std::max<int64_t>((int64_t)std::floor((pos[a][i] - g.origin[a]) / g.edge), 1);
        const int64_t key = (b[2] * g.dims[1] + b[1]) * g.dims[0] + b[0];
        g.next[i] = __atomic_exchange_n(&g.head[key], i, __ATOMIC_RELAXED);
    }
}

}  // namespace

// Advances `rows` (n x (x, y, z, diameter), float32, in place) by nsteps with
// `threads` OpenMP threads (0 = all); returns the seconds the steps took
// (conversion to and from float64 excluded).
extern "C" double ugcpu_steps(float *rows, uint32_t n, Params p, int nsteps, int threads) {
    if (threads > 0) omp_set_num_threads(threads);
    std::vector<double> pos[3], diam(n), f[3];
    for (int a = 0; a < 3; ++a) {
        pos[a].resize(n);
        f[a].resize(n);
    }
    for (uint32_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) pos[a][i] = rows[4 * (size_t)i + a];
        diam[i] = rows[4 * (size_t)i + 3];
    }
    const double k = p.k, gamma = p.gamma, m2 = 2.0 * (double)p.contact_margin;
    Grid g;
    const auto t0 = std::chrono::steady_clock::now();
    for (int s = 0; s < nsteps; ++s) {
        build_grid(pos, diam, p.contact_margin, g);
#pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t i = 0; i < (int64_t)n; ++i) {
            int64_t b[3];
            for (int a = 0; a < 3; ++a)
                b[a] = std::max<int64_t>((int64_t)std::floor((pos[a][i] - g.origin[a]) / g.edge), 1);
            const double ri = 0.5 * diam[i];
            double F[3] = {0.0, 0.0, 0.0};
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int64_t key = ((b[2] + dz) * g.dims[1] + (b[1] + dy)) * g.dims[0] + b[0] + dx;
                        for (int64_t j = g.head[key]; j >= 0; j = g.next[j]) {
                            if (j == i) continue;
                            const double h[3] = {pos[0][i] - pos[0][j], pos[1][i] - pos[1][j],
                                                 pos[2][i] - pos[2][j]};
                            const double d = std::sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
                            const double rj = 0.5 * diam[j];
                            const double delta = ri + rj + m2 - d;
                            if (!(delta > 0.0) || !(d > 0.0)) continue;
                            const double R = ri * rj / (ri + rj);
                            const double c = (k * delta - gamma * std::sqrt(R * delta)) / d;
                            for (int a = 0; a < 3; ++a) F[a] += c * h[a];
                        }
                    }
            for (int a = 0; a < 3; ++a) f[a][i] = F[a];
        }
#pragma omp parallel for
        for (int64_t i = 0; i < (int64_t)n; ++i) {
            const double Fn = std::sqrt(f[0][i] * f[0][i] + f[1][i] * f[1][i] + f[2][i] * f[2][i]);
            if (!(Fn > (double)p.adherence)) continue;
            const double m = (double)p.density * (M_PI / 6.0) * diam[i] * diam[i] * diam[i];
            double v[3], vn2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                v[a] = (double)p.dt / m * f[a][i];
                vn2 += v[a] * v[a];
            }
            const double vn = std::sqrt(vn2);
            const double scale = vn > (double)p.max_disp ? (double)p.max_disp / vn : 1.0;
            for (int a = 0; a < 3; ++a) pos[a][i] += v[a] * scale;
        }
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (uint32_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) rows[4 * (size_t)i + a] = (float)pos[a][i];
    return secs;
}

// Threads OpenMP would use by default.
extern "C" int ugcpu_max_threads() { return omp_get_max_threads(); }
