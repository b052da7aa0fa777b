// Symmetric pair evaluation (Newton's third law) of Eq. 1: the force entry
// ug_forces_symmetric and the step ug_step_pairs_once (k_sym + k_sym_move).
//
// Each agent walks only the forward half of its neighbourhood -- the three runs
// of the plane above (dz = +1), the run of the row above in its own plane
// (dz = 0, dy = +1), and the rest of its own run (the later agents of its box
// and the box after it) -- so every overlapping pair is found once, by its
// earlier agent.  The pair's force goes to both agents as 64-bit fixed-point
// integers (2^-32 units): integer sums do not depend on the order of the
// atomics, so the result is deterministic.  The same kernel with FORWARD =
// false walks all 27 boxes and adds only to its own agent, which gives the
// same bits (f_ji = -f_ij exactly in the float-float contact arithmetic, and
// rounding to fixed point is symmetric): the comparison that isolates what
// evaluating each pair once saves.  With WIN the four forward rows and the rest
// of the own row are cut to the agent's x-window (row_window), which holds all
// its contacts in that row, so the pairs found and the sums are the same.
#include <cuda_runtime.h>

#include "ug_internal.cuh"

namespace ug {

// Fixed point: 2^-32 force units in int64, so a sum holds |F| < 2^31 units.
// Each pair's components are checked against 2^30 (reported as UG_EBADSTATE);
// with the default constants and diameters ~10 a pair force (kappa delta -
// gamma sqrt(R delta)) is a few tens of units, so a sum stays far inside the
// range for any realistic number of overlapping neighbours.
constexpr float kFixScale = 4294967296.0f;           // 2^32
constexpr float kFixLimit = 1073741824.0f;            // |force component| < 2^30 per pair

__device__ __forceinline__ long long to_fix(float v) { return __float2ll_rn(v * kFixScale); }

// Candidates listed per agent between flushes: longer than the main sweep's
// lists, since a flush here costs three atomics per pair.
constexpr int kSymCap = 28;
struct SymList {
    uint32_t lst[kSymCap][32];
};

template <bool FORWARD, bool CHAINED, bool WIN>
__global__ void __launch_bounds__(128)
k_sym(const float4 *__restrict__ st, const uint32_t *__restrict__ start,
      const ug_grid_info *__restrict__ geo, SimArgs sa,
      unsigned long long *acc, int32_t *status, const uint32_t *__restrict__ skey) {
    __shared__ SymList wl[4];
    if (CHAINED) chain_begin();
    if (cta_failed(status)) return;
    const int lane = threadIdx.x & 31;
    SymList &w = wl[threadIdx.x >> 5];
    const uint32_t n = sa.n;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    // each lane with its own simulation's grid and constants (every pair lies
    // inside one simulation, so the forward walk never leaves it)
    bool uniform;
    const uint32_t sim = cta_sim(sa, blockIdx.x * blockDim.x, i, uniform);
    const ug_grid_info g = sim_geo(sa, geo, sim);
    const ug_params P = sim_params(sa, sim);
    const float m2 = 2.0f * P.contact_margin;
    const float4 me = valid ? __ldg(st + i) : make_float4(1e30f, 1e30f, 1e30f, 1.0f);
    uint32_t key = 0;
    if (valid) {
        int bx, by, bz;
        key = skey ? box_of_sort_key(__ldg(skey + i), g) : box_key(me, g, bx, by, bz);
    }
    const bool exact_diffs = __all_sync(kFull, !valid || far_from_origin(me, g.edge));
    const FilterRow fr = make_filter_row(me, m2);
    const float ri = 0.5f * me.w;
    const int ks = grid_shift(g);
    const uint32_t K = 1u << ks;
    const uint32_t row = (uint32_t)g.dims[0] << ks;
    const uint32_t plane = ((uint32_t)g.dims[0] * (uint32_t)g.dims[1]) << ks;
    static_assert(FORWARD || !WIN, "the windows serve the forward walk");
    AgentBox ab{};
    float slx = 0.f, sly = 0.f, slz = 0.f;
    if (WIN) {
        ab = agent_box(me, g, __frcp_rn(g.edge), P.contact_margin);
        slx = (float)(g.dims[0] + 2) * kWinSlack;
        sly = (float)(g.dims[1] + 2) * kWinSlack;
        slz = (float)(g.dims[2] + 2) * kWinSlack;
    }
    long long sx = 0, sy = 0, sz = 0;
    uint32_t np = 0;
    bool overflow = false;
    int cnt = 0;
    auto flush = [&]() {
        const int m = (int)__reduce_max_sync(kFull, (unsigned)cnt);
        for (int k = 0; k < m; ++k) {
            if (k >= cnt) continue;
            const uint32_t j = w.lst[k][lane];
            ContactGeo c;
            const float4 q = __ldg(st + j);
            const bool hit = exact_diffs ? contact_t<false>(me, ri, q, m2, c)
                                         : contact_t<true>(me, ri, q, m2, c);
            if (!hit) continue;
            const float coef = eq1_coef(ri, c.rb, c.rsum, c.delta, c.invd, P.k, P.gamma);
            const float fx = __fmul_rn(coef, c.hx), fy = __fmul_rn(coef, c.hy), fz = __fmul_rn(coef, c.hz);
            overflow |= !(fabsf(fx) < kFixLimit && fabsf(fy) < kFixLimit && fabsf(fz) < kFixLimit);
            const long long ax = to_fix(fx), ay = to_fix(fy), az = to_fix(fz);
            sx += ax;
            sy += ay;
            sz += az;
            ++np;
            if (FORWARD) {   // Newton's third law: the same pair pushes j the other way
                atomicAdd(acc + 4 * (size_t)j + 0, (unsigned long long)(-ax));
                atomicAdd(acc + 4 * (size_t)j + 1, (unsigned long long)(-ay));
                atomicAdd(acc + 4 * (size_t)j + 2, (unsigned long long)(-az));
                if (!CHAINED) atomicAdd(acc + 4 * (size_t)j + 3, 1ull);   // the step needs no counts
            }
        }
        cnt = 0;
    };
    // runs: FORWARD walks (dz = +1, dy = -1..1), (dz = 0, dy = +1) and the own
    // run after i; otherwise all 9 runs
    constexpr int kRuns = FORWARD ? 5 : 9;
#pragma unroll 1
    for (int r = 0; r < kRuns; ++r) {
        uint32_t b = valid ? i : 0u;
        int len = 0;
        if (valid && WIN) {
            // forward rows (dz, dy) = (1, -1), (1, 0), (1, 1), (0, 1), then the
            // own row after i, each cut to the agent's x-window
            const int dz = r < 3 ? 1 : 0;
            const int dy = r < 3 ? r - 1 : (r == 3 ? 1 : 0);
            int lo, hi;
            if (row_window(ab, dy, dz, sly, slz, slx, (float)K, (int)K, lo, hi)) {
                const uint32_t rb = key + (uint32_t)dz * plane + (uint32_t)dy * row -
                                    ((uint32_t)ab.bx << ks);
                b = r == 4 ? i + 1 : __ldg(start + rb + (uint32_t)lo);
                len = (int)(__ldg(start + rb + (uint32_t)hi + 1u) - b);
            }
            if (len <= 0) { len = 0; b = i; }
        } else if (valid) {
            if (FORWARD && r == 4) {
                b = i + 1;
                len = (int)(__ldg(start + key + 2u * K) - b);
            } else {
                const int dz = FORWARD ? (r < 3 ? 1 : 0) : r / 3 - 1;
                const int dy = FORWARD ? (r < 3 ? r - 1 : 1) : r % 3 - 1;
                const uint32_t kb = key + (uint32_t)dz * plane + (uint32_t)dy * row;
                b = __ldg(start + kb - K);
                len = (int)(__ldg(start + kb + 2u * K) - b);
            }
            if (len <= 0) { len = 0; b = i; }
        }
        const int last = max(len - 1, 0);
        const int lmax = (int)__reduce_max_sync(kFull, (unsigned)len);
        for (int t = 0; t < lmax; t += kSweepUnroll) {
#pragma unroll
            for (int u = 0; u < kSweepUnroll; ++u) {
                const uint32_t jc = b + (uint32_t)min(t + u, last);
                const float4 q = __ldg(st + jc);
                if ((t + u < len) & (jc != i) & prefilter(q, fr)) {
                    w.lst[cnt][lane] = jc;
                    ++cnt;
                }
            }
            if (__any_sync(kFull, cnt > kSymCap - kSweepUnroll)) flush();
        }
    }
    flush();
    if (overflow) set_status(status, UG_EBADSTATE);
    if (!valid) return;
    if (FORWARD && CHAINED) {
        // the step: the agent's own sums go to their own slots (no atomics),
        // the move kernel adds the other agents' contributions
        ulonglong2 *own = reinterpret_cast<ulonglong2 *>(acc + 4 * (size_t)n + 4 * (size_t)i);
        own[0] = make_ulonglong2((unsigned long long)sx, (unsigned long long)sy);
        own[1] = make_ulonglong2((unsigned long long)sz, 0ull);
    } else if (FORWARD) {
        atomicAdd(acc + 4 * (size_t)i + 0, (unsigned long long)sx);
        atomicAdd(acc + 4 * (size_t)i + 1, (unsigned long long)sy);
        atomicAdd(acc + 4 * (size_t)i + 2, (unsigned long long)sz);
        atomicAdd(acc + 4 * (size_t)i + 3, (unsigned long long)np);
    } else {
        acc[4 * (size_t)i + 0] = (unsigned long long)sx;
        acc[4 * (size_t)i + 1] = (unsigned long long)sy;
        acc[4 * (size_t)i + 2] = (unsigned long long)sz;
        acc[4 * (size_t)i + 3] = (unsigned long long)np;
    }
}

__global__ void __launch_bounds__(256)
k_sym_finish(const unsigned long long *__restrict__ acc, uint32_t n, float4 *__restrict__ force,
             int32_t *status) {
    if (cta_failed(status)) return;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float inv = 1.0f / kFixScale;
    force[i] = make_float4((float)(long long)acc[4 * (size_t)i + 0] * inv,
                           (float)(long long)acc[4 * (size_t)i + 1] * inv,
                           (float)(long long)acc[4 * (size_t)i + 2] * inv,
                           (float)acc[4 * (size_t)i + 3]);
}

// Move kernel of the symmetric step: the other agents' contributions plus the
// agent's own sums become F (the former cleared for the next step), then the
// Sec. III displacement moves the agent, the bounds of the moved rows
// accumulate, and the last CTA finalises the next step's grid.
__global__ void __launch_bounds__(256)
k_sym_move(const float4 *__restrict__ st, unsigned long long *acc, SimArgs sa, SweepOut out,
           int32_t *status) {
    __shared__ uint32_t s_red[32 * kBoundsWords];
    __shared__ FinalizeScratch fs;
    chain_begin();
    if (cta_failed(status)) return;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < sa.n;
    bool uniform;
    const uint32_t sim = cta_sim(sa, blockIdx.x * blockDim.x, i, uniform);
    const ug_params P = sim_params(sa, sim);
    uint32_t codes[8];
    float4 nw = make_float4(0.f, 0.f, 0.f, 1.f);
    if (valid) {
        const float inv = 1.0f / kFixScale;
        ulonglong2 *a2 = reinterpret_cast<ulonglong2 *>(acc + 4 * (size_t)i);
        const ulonglong2 *o2 = reinterpret_cast<const ulonglong2 *>(acc + 4 * (size_t)sa.n + 4 * (size_t)i);
        const ulonglong2 xy = a2[0], zc = a2[1], oxy = o2[0], ozc = o2[1];
        a2[0] = make_ulonglong2(0ull, 0ull);
        a2[1] = make_ulonglong2(0ull, 0ull);
        const float Fx = (float)(long long)(xy.x + oxy.x) * inv, Fy = (float)(long long)(xy.y + oxy.y) * inv,
                    Fz = (float)(long long)(zc.x + ozc.x) * inv;
        const float4 me = __ldg(st + i);
        bool mv, cp;
        const float3 u = displacement(Fx, Fy, Fz, me.w, P, &mv, &cp);
        nw = make_float4(me.x + u.x, me.y + u.y, me.z + u.z, me.w);
        out.state_out[i] = nw;
        if (out.force) out.force[i] = make_float4(Fx, Fy, Fz, (mv ? 1.f : 0.f) + (cp ? 2.f : 0.f));
        if (!row_ok(nw)) set_status(status, UG_EBADSTATE);
    }
    bounds_codes(nw, valid, codes);
    accumulate_bounds_codes(sa, codes, valid, sim, uniform, out.bounds, s_red, kBoundsWords);
    if (elect_last_cta(&out.ctrl->done))
        finalize_grid(sa, out.bounds, out.geo_next, out.ctrl, out.max_boxes, status, fs);
}

void launch_sym_step(const float4 *sorted, const uint32_t *start, const ug_grid_info *geo,
                     const SimArgs &sa, const SweepOut &out, unsigned long long *acc,
                     int32_t *status, cudaStream_t s, const uint32_t *skey, bool windowed) {
    const uint32_t n = sa.n;
    if (windowed)
        launch_chained(k_sym<true, true, true>, (unsigned)((n + 127) / 128), 128u, s, sorted, start,
                       geo, sa, acc, status, skey);
    else
        launch_chained(k_sym<true, true, false>, (unsigned)((n + 127) / 128), 128u, s, sorted, start,
                       geo, sa, acc, status, skey);
    launch_chained(k_sym_move, (unsigned)((n + 255) / 256), 256u, s, sorted, acc, sa, out, status);
}

int run_symmetric(bool forward, const float4 *sorted, const uint32_t *start, const ug_grid_info *geo,
                  uint32_t n, const ug_params &p, unsigned long long *acc, float4 *force,
                  int32_t *status, cudaStream_t s) {
    if (forward && cudaMemsetAsync(acc, 0, 32 * (size_t)n, s) != cudaSuccess) return UG_ECUDA;
    SimArgs sa{};
    sa.nsims = 1;
    sa.n = n;
    sa.pval = p;
    sa.bounds_copies = 1;
    sa.per_box_table = true;   // the caller's table from ug_grid_build
    const unsigned grid = (unsigned)((n + 127) / 128);
    if (forward)
        k_sym<true, false, false><<<grid, 128, 0, s>>>(sorted, start, geo, sa, acc, status, nullptr);
    else
        k_sym<false, false, false><<<grid, 128, 0, s>>>(sorted, start, geo, sa, acc, status, nullptr);
    k_sym_finish<<<(n + 255) / 256, 256, 0, s>>>(acc, n, force, status);
    return cudaGetLastError() == cudaSuccess ? UG_OK : UG_ECUDA;
}

}  // namespace ug
