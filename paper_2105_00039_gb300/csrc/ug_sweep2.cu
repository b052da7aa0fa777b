// Neighbour sweep with two agents per lane (Hesam et al., Sec. III and IV-A).
//
// Lane l of the grid handles the box-sorted agents 2l and 2l+1.  Consecutive
// agents usually share a box or sit in adjacent boxes of one row, so for each
// of the 9 neighbour rows the two agents' candidate runs merge into one run:
// every candidate row is loaded once and tested against both agents, which
// halves the per-candidate index, load and loop work of the one-agent-per-lane
// sweep.  A lane whose two agents lie too far apart in box order to merge walks
// the two 9-run sets one after the other.  k_sweep2<..., WIN> cuts each run to
// the agents' x-windows (see row_window); without WIN a run is the row's three
// boxes (the host picks, see windows_pay).  Runs are walked in
// warp lockstep (k_sweep2 concatenates the three runs of each neighbour plane,
// so the trip count is the warp's longest concatenation) with clamped indices
// and masks; neighbouring lanes read the same candidate rows at the same time,
// which the L1 serves once.  Candidates that pass the packed float32
// pre-filter go to per-agent lists, and the exact float-float contact test and
// Eq. 1 run in warp-converged batches (in k_sweep2 both agents' k-th entries in
// one FP32x2 pass, contact_eq1_x2).  k_sweep2 serves one simulation and leaves
// the next grid to k_finalize1;
// k_sweep2m serves many (a lane whose agents belong to different simulations
// walks them separately, each with its own simulation's grid and constants).
#include <cuda_runtime.h>

#include "ug_internal.cuh"

namespace ug {

// Candidates per agent between flushes: 24 in the one-simulation sweep (a
// mean of 8 contacts then rarely needs a flush before the end of the walk),
// 16 in the batched one.
constexpr int kListCap1 = 24;
constexpr int kListCap2 = 16;

template <int CAP>
struct __align__(16) WarpListsT {
    uint32_t lst[2][CAP][32];
};
using WarpLists1 = WarpListsT<kListCap1>;
using WarpLists2 = WarpListsT<kListCap2>;
static_assert(2 * sizeof(WarpLists2) >= sizeof(FinalizeScratch),
              "the epilogue reuses the lists of a CTA of 2 or more warps");

struct Accum {
    float sx, sy, sz, cx, cy, cz;
    uint32_t np;
};

__device__ __forceinline__ void add_contact(const float4 &me, const float4 &q, float m2,
                                            bool exact_diffs, const ug_params &P, Accum &a) {
    ContactGeo c;
    const float ri = 0.5f * me.w;
    const bool hit = exact_diffs ? contact_t<false>(me, ri, q, m2, c)
                                 : contact_t<true>(me, ri, q, m2, c);
    if (!hit) return;
    const float coef = eq1_coef(ri, c.rb, c.rsum, c.delta, c.invd, P.k, P.gamma);
    comp_add(a.sx, a.cx, __fmul_rn(coef, c.hx));
    comp_add(a.sy, a.cy, __fmul_rn(coef, c.hy));
    comp_add(a.sz, a.cz, __fmul_rn(coef, c.hz));
    ++a.np;
}

// The float32 pre-filter of one candidate row against both agents of a lane,
// packed across the two agents (element 0 of each pair is agent 0, element 1
// agent 1): three differences, the scaled contact distance, the squared
// centre distance (a multiply and two fused multiply-adds) and the squared
// contact distance, eight packed operations for both agents where two
// prefilter() calls take twelve.  Same band as prefilter().
struct FilterPair {
    float2 nx, ny, nz, s;
};
__device__ __forceinline__ FilterPair make_filter_pair(const float4 &a, const float4 &b, float m2) {
    FilterPair f;
    f.nx = make_float2(-a.x, -b.x);
    f.ny = make_float2(-a.y, -b.y);
    f.nz = make_float2(-a.z, -b.z);
    f.s = make_float2((0.5f * a.w + m2) * kFilterRoot, (0.5f * b.w + m2) * kFilterRoot);
    return f;
}
__device__ __forceinline__ void prefilter_pair(const float4 &q, const FilterPair &f, bool &p0,
                                               bool &p1) {
    const float2 dx = __fadd2_rn(make_float2(q.x, q.x), f.nx);
    const float2 dy = __fadd2_rn(make_float2(q.y, q.y), f.ny);
    const float2 dz = __fadd2_rn(make_float2(q.z, q.z), f.nz);
    const float h = 0.5f * kFilterRoot;
    const float2 sv = __ffma2_rn(make_float2(q.w, q.w), make_float2(h, h), f.s);
    float2 d2 = __fmul2_rn(dx, dx);
    d2 = __ffma2_rn(dy, dy, d2);
    d2 = __ffma2_rn(dz, dz, d2);
    const float2 s2 = __fmul2_rn(sv, sv);
    p0 = d2.x < s2.x;
    p1 = d2.y < s2.y;
}

// Exact contact test and Eq. 1 for the candidates listed since the last flush,
// warp-converged (every lane calls it; trip count = the warp's longest list,
// both agents' entries k in one pass).  DIFFS_EXACT: the warp's float32 centre
// differences are exact (far_from_origin), else they are formed with TwoSum.
template <bool DIFFS_EXACT>
__device__ __forceinline__ void flush_lists1(const float4 *__restrict__ st, const WarpLists1 *w,
                                             int c0, int c1, const float4 &me0, const float4 &me1,
                                             float m2, const ug_params &P, Accum &a0, Accum &a1) {
    const int lane = threadIdx.x & 31;
    const int m = (int)__reduce_max_sync(kFull, (unsigned)max(c0, c1));
    if (m == 0) return;
    const float2 ax = pk(me0.x, me1.x), ay = pk(me0.y, me1.y), az = pk(me0.z, me1.z);
    const float2 ra = pk(0.5f * me0.w, 0.5f * me1.w);
    const float2 kk = pk(P.k, P.k), gg = pk(P.gamma, P.gamma);
    float2 SX = pk(a0.sx, a1.sx), SY = pk(a0.sy, a1.sy), SZ = pk(a0.sz, a1.sz);
    float2 CX = pk(a0.cx, a1.cx), CY = pk(a0.cy, a1.cy), CZ = pk(a0.cz, a1.cz);
    for (int k = 0; k < m; ++k) {
        const bool h0 = k < c0, h1 = k < c1;
        const float4 q0 = __ldg(st + (h0 ? w->lst[0][k][lane] : 0u));   // row 0: a row that exists
        const float4 q1 = __ldg(st + (h1 ? w->lst[1][k][lane] : 0u));
        float2 hx, hy, hz, coef;
        bool t0, t1;
        contact_eq1_x2<DIFFS_EXACT>(ax, ay, az, ra, q0, q1, h0, h1, m2, kk, gg, hx, hy, hz, coef,
                                    t0, t1);
        const float2 cz = pk(t0 ? coef.x : 0.0f, t1 ? coef.y : 0.0f);
        float2 t, e;
        two_sum2(SX, mul2_unfused(cz, hx), t, e); SX = t; CX = add2(CX, e);
        two_sum2(SY, mul2_unfused(cz, hy), t, e); SY = t; CY = add2(CY, e);
        two_sum2(SZ, mul2_unfused(cz, hz), t, e); SZ = t; CZ = add2(CZ, e);
        a0.np += t0;
        a1.np += t1;
    }
    a0.sx = SX.x; a1.sx = SX.y; a0.sy = SY.x; a1.sy = SY.y; a0.sz = SZ.x; a1.sz = SZ.y;
    a0.cx = CX.x; a1.cx = CX.y; a0.cy = CY.x; a1.cy = CY.y; a0.cz = CZ.x; a1.cz = CZ.y;
}

// The same for the batched sweep, where the two agents may belong to different
// simulations; out of line with the difference mode a run-time argument, so
// that one copy of the long contact test serves its walk loops.
__device__ __noinline__ void flush_lists2m(const float4 *__restrict__ st, const WarpLists2 *w,
                                           int c0, int c1, float4 me0, float4 me1, float m20,
                                           float m21, bool exact_diffs, ug_params P0,
                                           ug_params P1, Accum *a0, Accum *a1) {
    const int lane = threadIdx.x & 31;
    const int m0 = (int)__reduce_max_sync(kFull, (unsigned)c0);
    for (int k = 0; k < m0; ++k)
        if (k < c0) add_contact(me0, __ldg(st + w->lst[0][k][lane]), m20, exact_diffs, P0, *a0);
    const int m1 = (int)__reduce_max_sync(kFull, (unsigned)c1);
    for (int k = 0; k < m1; ++k)
        if (k < c1) add_contact(me1, __ldg(st + w->lst[1][k][lane]), m21, exact_diffs, P1, *a1);
}

// The two agents' windows merge into one run per neighbour row, boxes
// [k0 - 1, k1 + 1] shifted by the row's offset (box keys; the table has
// K = 2^ks entries per box, so in table entries k0 - K .. k1 + 2K), when no two of the 9 merged
// runs can overlap: the 9 offsets are at least one x-row (dims_x boxes) apart,
// so runs of k1 - k0 + 3 boxes stay disjoint while k1 - k0 <= dims_x - 3.
// That holds for two agents of one x-row and for the usual pair that straddles
// a row end (the boxes between them are the two empty padding boxes).  As the
// runs are disjoint, the extra boxes a merged run covers lie outside both
// agents' 27-box neighbourhoods, so no contact is found (or counted twice)
// there.  The order in which an agent meets
// its contacts is the same merged or split: ascending within each run, runs in
// the same order.
__device__ __forceinline__ bool mergeable(uint32_t k0, uint32_t k1, uint32_t dx, int ks) {
    return k1 >= k0 && ((k1 - k0) >> ks) + 3u <= dx;
}

// The three runs of neighbour plane dz cut to the served agents' windows (the
// union of agent 0's and agent 1's where both are served): out[2r], out[2r+1]
// are the first and the end slot of row dy = r - 1 (equal when it holds no
// candidate).  Out of line, so that the walk's registers are not spent on it;
// the two agents' boxes (ab[0], ab[1]) are computed once per lane and kept in
// local memory.
__device__ __noinline__ void plane_windows(const AgentBox *ab, bool s0, bool s1, uint32_t k0,
                                           uint32_t k1, int dz, int d0, int d1, int d2, int ks,
                                           const uint32_t *__restrict__ start, uint32_t *out) {
    const uint32_t K = 1u << ks, R = (uint32_t)d0 << ks;
    const uint32_t plane = ((uint32_t)d0 * (uint32_t)d1) << ks;
    const float slx = (float)(d0 + 2) * kWinSlack, sly = (float)(d1 + 2) * kWinSlack;
    const float slz = (float)(d2 + 2) * kWinSlack;
    const AgentBox a0 = ab[0];
    const AgentBox a1 = ab[1];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int dy = r - 1;
        uint32_t wl = 0xffffffffu, wh = 0u;
        auto take = [&](const AgentBox &a, uint32_t key) {
            int l, h;
            if (!row_window(a, dy, dz, sly, slz, slx, (float)K, (int)K, l, h)) return;
            // the row's first table entry: the key's row shifted by (dy, dz)
            const uint32_t rb = key + (uint32_t)dz * plane + (uint32_t)dy * R - ((uint32_t)a.bx << ks);
            wl = min(wl, rb + (uint32_t)l);
            wh = max(wh, rb + (uint32_t)h + 1u);
        };
        if (s0) take(a0, k0);
        if (s1) take(a1, k1);
        const bool any = wl < wh;
        out[2 * r] = any ? __ldg(start + wl) : 0u;
        out[2 * r + 1] = any ? __ldg(start + wh) : 0u;
    }
}

// Six CTAs per SM: with 24-entry lists (24 KB a CTA of 128 threads) and the
// inlined flush, fewer resident warps and a larger L1 beat eight.
template <int MODE, int T, bool WIN>
__global__ void __launch_bounds__(T, 6)
k_sweep2(const float4 *__restrict__ st, const uint32_t *__restrict__ start,
         const ug_grid_info *__restrict__ geo, const uint32_t *__restrict__ skey, SimArgs sa,
         SweepOut out, int32_t *status) {
    __shared__ WarpLists1 wl[T / 32];
    chain_begin();
    if (cta_failed(status)) return;
    const int lane = threadIdx.x & 31;
    WarpLists1 &w = wl[threadIdx.x >> 5];
    const uint32_t n = sa.n;
    const uint32_t i0 = (blockIdx.x * T + threadIdx.x) * 2u, i1 = i0 + 1u;
    const bool v0 = i0 < n, v1 = i1 < n;
    const ug_params P = sim_params(sa, 0);   // the constants as a single or batched call passes them
    const ug_grid_info g = sim_geo(sa, geo, 0);
    const float m2 = 2.0f * P.contact_margin;
    const float4 far = make_float4(1e30f, 1e30f, 1e30f, 1.0f);
    const float4 me0 = v0 ? __ldg(st + i0) : far;
    const float4 me1 = v1 ? __ldg(st + i1) : far;
    const int ks = grid_shift(g);
    const uint32_t dx = (uint32_t)g.dims[0], dimy = (uint32_t)g.dims[1];
    const uint32_t K = 1u << ks, R = dx << ks;                   // table entries per box, per row
    const uint32_t plane = ((uint32_t)g.dims[0] * (uint32_t)g.dims[1]) << ks;
    uint32_t k0 = 0, k1 = 0;
    if (v0) {
        int bx, by, bz;
        k0 = skey ? box_of_sort_key(__ldg(skey + i0), g) : box_key(me0, g, bx, by, bz);
        k1 = k0;
        if (v1) k1 = skey ? box_of_sort_key(__ldg(skey + i1), g) : box_key(me1, g, bx, by, bz);
    }
    const bool split = v1 && !mergeable(k0, k1, dx, ks);
    const bool exact_diffs =
        __all_sync(kFull, (!v0 || far_from_origin(me0, g.edge)) && (!v1 || far_from_origin(me1, g.edge)));
    const FilterPair fp = make_filter_pair(me0, me1, m2);
    AgentBox abox[2];
    if (WIN) {
        const float inv_e = __frcp_rn(g.edge);
        abox[0] = agent_box(me0, g, inv_e, P.contact_margin);
        abox[1] = agent_box(me1, g, inv_e, P.contact_margin);
    }
    Accum acc[2] = {{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u}, {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u}};
    int c0 = 0, c1 = 0;
    auto flush = [&]() {
        if (exact_diffs) flush_lists1<true>(st, &w, c0, c1, me0, me1, m2, P, acc[0], acc[1]);
        else flush_lists1<false>(st, &w, c0, c1, me0, me1, m2, P, acc[0], acc[1]);
        c0 = 0;
        c1 = 0;
    };
    // One lockstep walk over candidates [0, len) of this lane, candidate t being
    // row index_of(t) (t clamped into the lane's range, masked when t >= len);
    // four candidates per iteration keep four row loads in flight per lane.
    constexpr int kWalkUnroll = 4;
    auto walk = [&](int len, int lmax, bool s0, bool s1, auto index_of) {
        const int last = max(len - 1, 0);
        for (int t = 0; t < lmax; t += kWalkUnroll) {
#pragma unroll
            for (int u = 0; u < kWalkUnroll; ++u) {
                const uint32_t jc = index_of(min(t + u, last));
                const float4 q = __ldg(st + jc);
                const bool in = t + u < len;
                bool p0, p1;
                prefilter_pair(q, fp, p0, p1);
                if (in & s0 & (jc != i0) & p0) {
                    w.lst[0][c0][lane] = jc;
                    ++c0;
                }
                if (in & s1 & (jc != i1) & p1) {
                    w.lst[1][c1][lane] = jc;
                    ++c1;
                }
            }
            if (__any_sync(kFull, max(c0, c1) > kListCap1 - kWalkUnroll)) flush();
        }
    };
    // The 9 runs come as 3 neighbour planes (dz) of 3 runs (dy = -1, 0, +1),
    // and a warp walks each plane's three runs as one sequence: candidate t of
    // a lane is row t + d0 while t < e1, t + d1 while t < e2, else t + d2.  The
    // trip count is then the warp's longest concatenation rather than the sum
    // of its longest runs, which pays where runs are short and uneven (sparse
    // grids); every agent meets its candidates in the same order as run by
    // run.  Planes 0..2 serve both agents (or agent 0 alone when split), 3..5
    // agent 1 when split.
    const int ngroups = __any_sync(kFull, split) ? 6 : 3;
#pragma unroll 1
    for (int gi = 0; gi < ngroups; ++gi) {
        const int dz = (gi < 3 ? gi : gi - 3) - 1;
        bool s0 = false, s1 = false;
        uint32_t d0 = v0 ? i0 : 0u, d1 = d0, d2 = d0;   // a row that exists when len == 0
        int e1 = 0, e2 = 0, len = 0;
        if (v0 && (gi < 3 || split)) {
            uint32_t lo, hi;
            if (!split) { lo = k0; hi = k1; s0 = true; s1 = v1; }
            else if (gi < 3) { lo = k0; hi = k0; s0 = true; }
            else { lo = k1; hi = k1; s1 = true; }
            uint32_t a0, x0, a1, x1, a2, x2;
            if (WIN) {
                uint32_t b6[6];
                plane_windows(abox, s0, s1, k0, k1, dz, g.dims[0], g.dims[1], g.dims[2], ks, start,
                              b6);
                a0 = b6[0]; x0 = b6[1]; a1 = b6[2]; x1 = b6[3]; a2 = b6[4]; x2 = b6[5];
            } else {
                const uint32_t lz = lo + (uint32_t)dz * plane, hz = hi + (uint32_t)dz * plane;
                a0 = __ldg(start + lz - R - K); x0 = __ldg(start + hz - R + 2u * K);
                a1 = __ldg(start + lz - K); x1 = __ldg(start + hz + 2u * K);
                a2 = __ldg(start + lz + R - K); x2 = __ldg(start + hz + R + 2u * K);
            }
            e1 = (int)(x0 - a0);
            e2 = e1 + (int)(x1 - a1);
            len = e2 + (int)(x2 - a2);
            if (len > 0) {
                d0 = a0;
                d1 = a1 - (uint32_t)e1;
                d2 = a2 - (uint32_t)e2;
            }
        }
        walk(len, (int)__reduce_max_sync(kFull, (unsigned)len), s0, s1, [&](int tt) {
            return (uint32_t)tt + (tt < e1 ? d0 : (tt < e2 ? d1 : d2));
        });
    }
    flush();

    const Accum &a0 = acc[0], &a1 = acc[1];
    const float3 F0 = make_float3(a0.sx + a0.cx, a0.sy + a0.cy, a0.sz + a0.cz);
    const float3 F1 = make_float3(a1.sx + a1.cx, a1.sy + a1.cy, a1.sz + a1.cz);
    if (MODE == kSweepForce) {
        if (v0) out.force[i0] = make_float4(F0.x, F0.y, F0.z, (float)a0.np);
        if (v1) out.force[i1] = make_float4(F1.x, F1.y, F1.z, (float)a1.np);
        return;
    }
    // fused step: Sec. III adherence / integration / cap, then move
    uint32_t codes[8], c2[8];
    float4 n0 = me0, n1 = me1;
    if (v0) {
        bool mv, cp;
        const float3 u = displacement(F0.x, F0.y, F0.z, me0.w, P, &mv, &cp);
        n0 = make_float4(me0.x + u.x, me0.y + u.y, me0.z + u.z, me0.w);
        out.state_out[i0] = n0;
        if (out.force) out.force[i0] = make_float4(F0.x, F0.y, F0.z, (mv ? 1.f : 0.f) + (cp ? 2.f : 0.f));
        if (!row_ok(n0)) set_status(status, UG_EBADSTATE);
    }
    if (v1) {
        bool mv, cp;
        const float3 u = displacement(F1.x, F1.y, F1.z, me1.w, P, &mv, &cp);
        n1 = make_float4(me1.x + u.x, me1.y + u.y, me1.z + u.z, me1.w);
        out.state_out[i1] = n1;
        if (out.force) out.force[i1] = make_float4(F1.x, F1.y, F1.z, (mv ? 1.f : 0.f) + (cp ? 2.f : 0.f));
        if (!row_ok(n1)) set_status(status, UG_EBADSTATE);
    }
    bounds_codes(n0, v0, codes);
    bounds_codes(n1, v1, c2);
#pragma unroll
    for (int k = 0; k < 8; ++k) codes[k] = max(codes[k], c2[k]);
    // the epilogue's scratch lives in the warps' list memory, no longer needed:
    // each warp's 8 bounds words in its own lists, the last CTA's grid
    // finalisation across all of them
    // each warp maximises its codes into one copy of the bounds accumulators
    // (no CTA barrier: a warp that finishes early does not wait for the
    // others); k_finalize1 turns them into the next grid
    const uint32_t copy = (blockIdx.x * (T / 32) + (threadIdx.x >> 5)) % sa.bounds_copies;
    uint32_t mine = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t m = __reduce_max_sync(kFull, codes[k]);
        if (lane == k) mine = m;
    }
    if (lane < 8 && mine) atomicMax(&out.bounds[(size_t)copy * kBoundsWords + lane], mine);
}

// The next step's grid of one simulation from the bounds k_sweep2 accumulated
// (finalize_grid is the code the other sweeps' last CTA runs).  256 threads:
// one read of the kBoundsCopiesSingle x kBoundsWords accumulators each.
__global__ void __launch_bounds__(256)
k_finalize1(SimArgs sa, uint32_t *bounds, ug_grid_info *geo, Ctrl *ctrl, uint32_t max_boxes,
            int32_t *status) {
    __shared__ FinalizeScratch fs;
    chain_begin();
    finalize_grid(sa, bounds, geo, ctrl, max_boxes, status, fs);
}

template <int MODE, int T, bool MULTI>
__global__ void __launch_bounds__(T, (MODE == kSweepStep && MULTI) ? 7 : 8)
k_sweep2m(const float4 *__restrict__ st, const uint32_t *__restrict__ start,
         const ug_grid_info *__restrict__ geo, const uint32_t *__restrict__ skey, SimArgs sa,
         SweepOut out, int32_t *status) {
    __shared__ WarpLists2 wl[T / 32];
    __shared__ uint32_t s_sims[2];
    chain_begin();
    if (cta_failed(status)) return;
    const int lane = threadIdx.x & 31;
    WarpLists2 &w = wl[threadIdx.x >> 5];
    const uint32_t n = sa.n;
    const uint32_t first = blockIdx.x * T * 2u;
    const uint32_t i0 = first + threadIdx.x * 2u, i1 = i0 + 1u;
    const bool v0 = i0 < n, v1 = i1 < n;
    // simulations of the two agents (one lookup per CTA when the CTA's agents share one)
    if (MULTI) {
        if (threadIdx.x == 0) {
            s_sims[0] = find_sim(sa, first);
            s_sims[1] = find_sim(sa, min(first + 2u * T, n) - 1u);
        }
        __syncthreads();
    }
    const bool uniform = !MULTI || s_sims[0] == s_sims[1];
    const uint32_t s0 = !MULTI ? 0u : uniform ? s_sims[0] : find_sim(sa, min(i0, n - 1u));
    const uint32_t s1 = !MULTI ? 0u : uniform ? s_sims[0] : find_sim(sa, min(i1, n - 1u));
    const ug_params P0 = sim_params(sa, s0);
    const ug_params P1 = s1 == s0 ? P0 : sim_params(sa, s1);
    const ug_grid_info g0 = sim_geo(sa, geo, s0);
    const ug_grid_info g1 = s1 == s0 ? g0 : sim_geo(sa, geo, s1);
    const float m20 = 2.0f * P0.contact_margin, m21 = 2.0f * P1.contact_margin;
    const float4 far = make_float4(1e30f, 1e30f, 1e30f, 1.0f);
    const float4 me0 = v0 ? __ldg(st + i0) : far;
    const float4 me1 = v1 ? __ldg(st + i1) : far;
    uint32_t k0 = 0, k1 = 0;
    if (v0) {
        int bx, by, bz;
        k0 = skey ? box_of_sort_key(__ldg(skey + i0), g0) : box_key(me0, g0, bx, by, bz);
        k1 = k0;
        if (v1) k1 = skey ? box_of_sort_key(__ldg(skey + i1), g1) : box_key(me1, g1, bx, by, bz);
    }
    const bool split = v1 && (s1 != s0 || !mergeable(k0, k1, (uint32_t)g0.dims[0], grid_shift(g0)));
    const bool exact_diffs = __all_sync(kFull, (!v0 || far_from_origin(me0, g0.edge)) &&
                                                   (!v1 || far_from_origin(me1, g1.edge)));
    const FilterRow f0 = make_filter_row(me0, m20), f1 = make_filter_row(me1, m21);
    Accum acc[2] = {{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u}, {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u}};
    Accum &a0 = acc[0], &a1 = acc[1];
    int c0 = 0, c1 = 0;
    auto flush = [&]() {
        flush_lists2m(st, &w, c0, c1, me0, me1, m20, m21, exact_diffs, P0, P1, &acc[0], &acc[1]);
        c0 = 0;
        c1 = 0;
    };
    constexpr int kWalkUnroll = 4;   // candidates per walk iteration (row loads in flight per lane)
    const int nruns = __any_sync(kFull, split) ? 18 : 9;
#pragma unroll 1
    for (int r = 0; r < nruns; ++r) {
        // runs 0..8 serve both agents (or agent 0 alone when split), 9..17 agent 1 when split
        const int rr = r < 9 ? r : r - 9;
        bool s0on = false, s1on = false;
        uint32_t b = v0 ? i0 : 0u;     // a row that exists; masked off when len == 0
        int len = 0;
        if (v0 && (r < 9 || split)) {
            uint32_t lo, hi;
            const ug_grid_info &g = r < 9 ? g0 : g1;
            if (!split) { lo = k0; hi = k1; s0on = true; s1on = v1; }
            else if (r < 9) { lo = k0; hi = k0; s0on = true; }
            else { lo = k1; hi = k1; s1on = true; }
            const int ks = grid_shift(g);
            const uint32_t K = 1u << ks;
            const uint32_t off = ((uint32_t)(rr / 3 - 1) * (uint32_t)g.dims[0] * (uint32_t)g.dims[1] +
                                  (uint32_t)(rr % 3 - 1) * (uint32_t)g.dims[0]) << ks;
            // indices in 32-bit arithmetic first: off may stand for a negative offset
            const uint32_t ib = lo + off - K, ie = hi + off + 2u * K;
            b = __ldg(start + ib);
            len = (int)(__ldg(start + ie) - b);
            if (len == 0) b = i0;
        }
        const int last = max(len - 1, 0);
        const int lmax = (int)__reduce_max_sync(kFull, (unsigned)len);
        for (int t = 0; t < lmax; t += kWalkUnroll) {
#pragma unroll
            for (int u = 0; u < kWalkUnroll; ++u) {
                const uint32_t jc = b + (uint32_t)min(t + u, last);
                const float4 q = __ldg(st + jc);
                const bool in = t + u < len;
                if (in & s0on & (jc != i0) & prefilter(q, f0)) {
                    w.lst[0][c0][lane] = jc;
                    ++c0;
                }
                if (in & s1on & (jc != i1) & prefilter(q, f1)) {
                    w.lst[1][c1][lane] = jc;
                    ++c1;
                }
            }
            if (__any_sync(kFull, max(c0, c1) > kListCap2 - kWalkUnroll)) flush();
        }
    }
    flush();

    const float3 F0 = make_float3(a0.sx + a0.cx, a0.sy + a0.cy, a0.sz + a0.cz);
    const float3 F1 = make_float3(a1.sx + a1.cx, a1.sy + a1.cy, a1.sz + a1.cz);
    if (MODE == kSweepForce) {
        if (v0) out.force[i0] = make_float4(F0.x, F0.y, F0.z, (float)a0.np);
        if (v1) out.force[i1] = make_float4(F1.x, F1.y, F1.z, (float)a1.np);
        return;
    }
    // fused step: Sec. III adherence / integration / cap, then move
    uint32_t codes[8], c2[8];
    float4 n0 = me0, n1 = me1;
    if (v0) {
        bool mv, cp;
        const float3 u = displacement(F0.x, F0.y, F0.z, me0.w, P0, &mv, &cp);
        n0 = make_float4(me0.x + u.x, me0.y + u.y, me0.z + u.z, me0.w);
        out.state_out[i0] = n0;
        if (out.force) out.force[i0] = make_float4(F0.x, F0.y, F0.z, (mv ? 1.f : 0.f) + (cp ? 2.f : 0.f));
        if (!row_ok(n0)) set_status(status, UG_EBADSTATE);
    }
    if (v1) {
        bool mv, cp;
        const float3 u = displacement(F1.x, F1.y, F1.z, me1.w, P1, &mv, &cp);
        n1 = make_float4(me1.x + u.x, me1.y + u.y, me1.z + u.z, me1.w);
        out.state_out[i1] = n1;
        if (out.force) out.force[i1] = make_float4(F1.x, F1.y, F1.z, (mv ? 1.f : 0.f) + (cp ? 2.f : 0.f));
        if (!row_ok(n1)) set_status(status, UG_EBADSTATE);
    }
    bounds_codes(n0, v0, codes);
    bounds_codes(n1, v1, c2);
    if (uniform) {
#pragma unroll
        for (int k = 0; k < 8; ++k) codes[k] = max(codes[k], c2[k]);
        accumulate_bounds_codes(sa, codes, v0, s0, true, out.bounds, &wl[0].lst[0][0][0],
                                sizeof(WarpLists2) / 4);
    } else {
        accumulate_bounds_codes(sa, codes, v0, s0, false, out.bounds, nullptr, 0u);
        accumulate_bounds_codes(sa, c2, v1, s1, false, out.bounds, nullptr, 0u);
    }
    if (elect_last_cta(&out.ctrl->done))
        finalize_grid(sa, out.bounds, out.geo_next, out.ctrl, out.max_boxes, status,
                      *reinterpret_cast<FinalizeScratch *>(wl));
}

void launch_sweep2(int mode, const float4 *sorted, const uint32_t *start, const ug_grid_info *geo,
                   const SimArgs &sa, const SweepOut &out, int32_t *status, cudaStream_t s,
                   const uint32_t *skey, bool windowed) {
    constexpr int T = 128;
    const unsigned grid = (unsigned)((sa.n + 2 * T - 1) / (2 * T));
    if (sa.nsims > 1) {
        if (mode == kSweepForce)
            launch_chained(k_sweep2m<kSweepForce, T, true>, grid, T, s, sorted, start, geo, skey, sa,
                           out, status);
        else
            launch_chained(k_sweep2m<kSweepStep, T, true>, grid, T, s, sorted, start, geo, skey, sa,
                           out, status);
    } else if (windowed) {
        if (mode == kSweepForce)
            launch_chained(k_sweep2<kSweepForce, T, true>, grid, T, s, sorted, start, geo, skey, sa,
                           out, status);
        else {
            launch_chained(k_sweep2<kSweepStep, T, true>, grid, T, s, sorted, start, geo, skey, sa,
                           out, status);
            launch_chained(k_finalize1, 1, 256, s, sa, out.bounds, out.geo_next, out.ctrl,
                           out.max_boxes, status);
        }
    } else {
        if (mode == kSweepForce)
            launch_chained(k_sweep2<kSweepForce, T, false>, grid, T, s, sorted, start, geo, skey, sa,
                           out, status);
        else {
            launch_chained(k_sweep2<kSweepStep, T, false>, grid, T, s, sorted, start, geo, skey, sa,
                           out, status);
            launch_chained(k_finalize1, 1, 256, s, sa, out.bounds, out.geo_next, out.ctrl,
                           out.max_boxes, status);
        }
    }
}

}  // namespace ug
