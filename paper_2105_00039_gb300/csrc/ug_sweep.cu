// Neighbour sweep and Eq. 1 (Hesam et al., Sec. III and IV-A), GB300 design.
//
// One thread per box-sorted agent.  With boxes numbered x-fastest, the 27
// neighbour boxes are 9 contiguous runs of 3 boxes (one per (dy, dz) row), so
// an agent's candidates are 9 slices of the sorted state; consecutive threads
// sit in the same or adjacent boxes and read the same slices, which the L1
// serves as broadcasts.  The 9 runs are walked as one flattened loop so that a
// warp's trip count is the largest candidate count of its lanes rather than
// the sum of per-run maxima.
//
// Two passes per agent keep the warp converged:
//   filter  a cheap float32 distance test (with a 2^-16 relative safety band,
//           so no true contact is dropped) appends candidate indices to a
//           per-lane list in shared memory;
//   refine  whenever a lane's list is full (warp vote) or the candidates are
//           exhausted, every lane evaluates its listed pairs with the exact
//           float-float contact test and Eq. 1, accumulating with TwoSum.
// Without the split, the expensive exact path would run in almost every
// iteration because some lane of the warp nearly always has a contact.
//
// Modes: forces only; the fused step (displacement, move, next step's bounds
// and grid geometry from the last CTA); or the contact list itself.
#include <cuda_runtime.h>

#include "ug_internal.cuh"

namespace ug {

// ------------------------------------------------------------------ staged traversal
// A warp's 32 consecutive agents lie in one to a few rows of boxes.  For each of
// those rows (at most kStageMaxRows) the warp copies the 9 neighbouring row
// segments that cover its agents' neighbourhoods, boxes [x_lo - 1, x_hi + 1],
// from the sorted rows into shared memory with coalesced cp.async, then every
// lane walks its own 9 runs inside the staged copy.  Returns false (nothing
// done) when the staged rows would not fit; the caller then walks global memory.
constexpr int kStageRows = 384;
constexpr int kStageList = 20;
constexpr int kStageMaxRows = 3;

struct WarpStaged {
    float4 rows[kStageRows];
    uint32_t runs[9][32];            // begin | end << 16, offsets into rows
    uint16_t lst[kStageList][32];
};
union WarpSmem {
    WarpLists gl;
    WarpStaged sg;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <typename Fn>
__device__ __forceinline__ bool sweep_staged(const float4 *__restrict__ st,
                                             const uint32_t *__restrict__ start,
                                             const ug_grid_info &g, uint32_t i, bool valid,
                                             const float4 &me_in, uint32_t key, float m2,
                                             WarpStaged &w, Fn &&fn) {
    const int lane = threadIdx.x & 31;
    const unsigned vmask = __ballot_sync(kFull, valid);
    if (vmask == 0u) return true;
    const int last_valid = 31 - __clz(vmask);
    const uint32_t dx = (uint32_t)g.dims[0];
    // invalid lanes (past n) take the last valid lane's box so that they add no row
    const uint32_t k = __shfl_sync(kFull, key, valid ? lane : last_valid);
    const int ks = grid_shift(g);
    const uint32_t K = 1u << ks;
    const uint32_t rel = (k - g.box_base) >> ks;
    const uint32_t row = rel / dx;
    const int bx = (int)(rel - row * dx);
    const uint32_t prev = __shfl_up_sync(kFull, row, 1);
    const unsigned heads = __ballot_sync(kFull, lane == 0 || prev != row);
    const int R = __popc(heads);
    if (R > kStageMaxRows) return false;
    const int myrow = __popc(heads & (0xffffffffu >> (31 - lane))) - 1;
    // lane s < 9R describes segment s = (warp row s / 9, neighbour row s % 9)
    const int sk = min(lane / 9, R - 1), sm = lane % 9;
    const int hl = (int)__fns(heads, 0, sk + 1);
    const int ll = sk + 1 < R ? (int)__fns(heads, 0, sk + 2) - 1 : last_valid;
    const uint32_t srow = __shfl_sync(kFull, row, hl);
    const int lo = __shfl_sync(kFull, bx, hl), hi = __shfl_sync(kFull, bx, ll);
    uint32_t sbeg = 0, slen = 0;
    if (lane < 9 * R) {
        const int dz = sm / 3 - 1, dy = sm % 3 - 1;
        const uint32_t kr = g.box_base + (((uint32_t)((int)srow + dz * g.dims[1] + dy) * dx) << ks);
        sbeg = __ldg(start + kr + ((uint32_t)(lo - 1) << ks));
        slen = __ldg(start + kr + ((uint32_t)(hi + 2) << ks)) - sbeg;
    }
    uint32_t soff = slen;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, soff, o);
        if (lane >= o) soff += y;
    }
    const uint32_t total_rows = __shfl_sync(kFull, soff, 31);
    soff -= slen;
    if (total_rows > (uint32_t)kStageRows) return false;
    for (int sg = 0; sg < 9 * R; ++sg) {
        const uint32_t b = __shfl_sync(kFull, sbeg, sg), o = __shfl_sync(kFull, soff, sg);
        const uint32_t L = __shfl_sync(kFull, slen, sg);
        for (uint32_t q = lane; q < L; q += 32) cp_async16(&w.rows[o + q], st + b + q);
    }
    // this lane's runs, as offsets into the staged rows (an empty run points
    // at the lane's own row, which the j != i test rejects)
    const float4 me = valid ? me_in : make_float4(1e30f, 1e30f, 1e30f, 1.f);
    const uint32_t plane = ((uint32_t)g.dims[0] * (uint32_t)g.dims[1]) << ks, rowk = dx << ks;
    uint32_t self = 0;
    {
        const uint32_t b4 = __shfl_sync(kFull, sbeg, myrow * 9 + 4);
        const uint32_t o4 = __shfl_sync(kFull, soff, myrow * 9 + 4);
        if (valid) self = o4 + (i - b4);
    }
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const int sg = myrow * 9 + r;
        const uint32_t b = __shfl_sync(kFull, sbeg, sg), o = __shfl_sync(kFull, soff, sg);
        uint32_t packed = self | (self << 16);
        if (valid) {
            const uint32_t kb = key + (uint32_t)(r / 3 - 1) * plane + (uint32_t)(r % 3 - 1) * rowk;
            const uint32_t rb = __ldg(start + kb - K), re = __ldg(start + kb + 2u * K);
            if (re > rb) packed = (o + (rb - b)) | ((o + (re - b)) << 16);
        }
        w.runs[r][lane] = packed;
    }
    cp_async_wait_all();
    __syncwarp();
    const FilterRow fr = make_filter_row(me, m2);
    int cnt = 0;
    auto flush = [&]() {
        const int m = (int)__reduce_max_sync(kFull, (unsigned)cnt);
        for (int kk = 0; kk < m; ++kk) {
            if (kk < cnt) fn(w.rows[w.lst[kk][lane]]);
        }
        cnt = 0;
    };
#pragma unroll 1
    for (int r = 0; r < 9; ++r) {
        const uint32_t c = w.runs[r][lane];
        const uint32_t b = c & 0xffffu;
        const int len = (int)(c >> 16) - (int)b;
        const int last = max(len - 1, 0);
        const int lmax = (int)__reduce_max_sync(kFull, (unsigned)len);
        for (int t = 0; t < lmax; t += kSweepUnroll) {
#pragma unroll
            for (int u = 0; u < kSweepUnroll; ++u) {
                const uint32_t jc = b + (uint32_t)min(t + u, last);
                const float4 cur = w.rows[jc];
                if ((t + u < len) & (jc != self) & prefilter(cur, fr)) {
                    w.lst[cnt][lane] = (uint16_t)jc;
                    ++cnt;
                }
            }
            if (__any_sync(kFull, cnt > kStageList - kSweepUnroll)) flush();
        }
    }
    flush();
    __syncwarp();
    return true;
}

template <int MODE, int T>
__global__ void __launch_bounds__(T)
k_sweep(const float4 *__restrict__ st, const uint32_t *__restrict__ start,
        const ug_grid_info *__restrict__ geo, const uint32_t *__restrict__ skey, SimArgs sa,
        SweepOut out, int32_t *status) {
    __shared__ WarpSmem wsm[T / 32];
    chain_begin();
    if (cta_failed(status)) return;
    const uint32_t first = blockIdx.x * T;
    const uint32_t i = first + threadIdx.x;
    const bool valid = i < sa.n;
    bool uniform;
    const uint32_t sim = cta_sim(sa, first, i, uniform);
    const ug_params P = sim_params(sa, sim);
    const ug_grid_info g = sim_geo(sa, geo, sim);
    const float m2 = 2.0f * P.contact_margin;
    WarpSmem &ws = wsm[threadIdx.x >> 5];

    const float4 me = valid ? __ldg(st + i) : make_float4(0.f, 0.f, 0.f, 1.f);
    const float ri = 0.5f * me.w;
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    uint32_t np = 0;
    // filtered candidates lie within e (+ rounding) of row i: if every lane of
    // the warp is far from the coordinate planes their differences are exact
    const bool exact_diffs = __all_sync(kFull, !valid || far_from_origin(me, g.edge));
    auto on_candidate = [&](const float4 &q) -> bool {
        ContactGeo c;
        const bool hit = exact_diffs ? contact_t<false>(me, ri, q, m2, c)
                                     : contact_t<true>(me, ri, q, m2, c);
        if (!hit) return false;
        if (MODE != kSweepPairs) {
            const float coef = eq1_coef(ri, c.rb, c.rsum, c.delta, c.invd, P.k, P.gamma);
            comp_add(sx, cx, __fmul_rn(coef, c.hx));
            comp_add(sy, cy, __fmul_rn(coef, c.hy));
            comp_add(sz, cz, __fmul_rn(coef, c.hz));
        }
        ++np;
        return true;
    };
    bool done = false;
    // a warp spanning two simulations walks global memory (batched boundaries)
    const bool warp_one_sim = uniform || __all_sync(kFull, sim == __shfl_sync(kFull, sim, 0));
    if (MODE != kSweepPairs && warp_one_sim) {
        uint32_t key_i = 0u;
        if (valid) {
            if (skey != nullptr) {
                key_i = box_of_sort_key(__ldg(skey + i), g);
            } else {
                int bx, by, bz;
                key_i = box_key(me, g, bx, by, bz);
            }
        }
        done = sweep_staged(st, start, g, i, valid, me, key_i, m2, ws.sg,
                            [&](const float4 &q) { on_candidate(q); });
    }
    if (!done) {
        const uint32_t key_i = (skey != nullptr && valid) ? box_of_sort_key(__ldg(skey + i), g) : 0xffffffffu;
        sweep_neighbours(st, start, g, i, valid, me, key_i, m2, ws.gl,
                         [&](uint32_t jj, const float4 &q) {
            const uint32_t before = np;
            on_candidate(q);
            if (MODE == kSweepPairs && np != before && before < out.max_per_agent)
                out.nbr[(size_t)i * out.max_per_agent + before] = jj;
        });
    }

    if (MODE == kSweepPairs) {
        if (valid) {
            out.pair_count[i] = np;
            if (np > out.max_per_agent) set_status(status, UG_ECAPACITY);
        }
        return;
    }
    const float Fx = sx + cx, Fy = sy + cy, Fz = sz + cz;
    if (MODE == kSweepForce) {
        if (valid) out.force[i] = make_float4(Fx, Fy, Fz, (float)np);
        return;
    }
    // fused step: Sec. III adherence / integration / cap, then move
    float4 nw = me;
    if (valid) {
        bool moving, capped;
        const float3 u = displacement(Fx, Fy, Fz, me.w, P, &moving, &capped);
        nw = make_float4(me.x + u.x, me.y + u.y, me.z + u.z, me.w);
        out.state_out[i] = nw;
        if (out.force) out.force[i] = make_float4(Fx, Fy, Fz, (moving ? 1.f : 0.f) + (capped ? 2.f : 0.f));
    }
    accumulate_bounds(sa, nw, valid, sim, uniform, out.bounds, status);
    __shared__ FinalizeScratch fs;
    if (elect_last_cta(&out.ctrl->done))
        finalize_grid(sa, out.bounds, out.geo_next, out.ctrl, out.max_boxes, status, fs);
}

template <int MODE>
static void launch_mode(const float4 *sorted, const uint32_t *start, const ug_grid_info *geo,
                        const SimArgs &sa, const SweepOut &out, int block, int32_t *status,
                        cudaStream_t s, const uint32_t *skey) {
    if (block == 64)
        launch_chained(k_sweep<MODE, 64>, (sa.n + 63) / 64, 64u, s, sorted, start, geo, skey, sa,
                       out, status);
    else
        launch_chained(k_sweep<MODE, 128>, (sa.n + 127) / 128, 128u, s, sorted, start, geo, skey,
                       sa, out, status);
}

void launch_sweep(int mode, const float4 *sorted, const uint32_t *start, const ug_grid_info *geo,
                  const SimArgs &sa, const SweepOut &out, int block, int32_t *status,
                  cudaStream_t s, const uint32_t *skey) {
    if (mode == kSweepForce)
        launch_mode<kSweepForce>(sorted, start, geo, sa, out, block, status, s, skey);
    else if (mode == kSweepStep)
        launch_mode<kSweepStep>(sorted, start, geo, sa, out, block, status, s, skey);
    else
        launch_mode<kSweepPairs>(sorted, start, geo, sa, out, block, status, s, skey);
}

// ------------------------------------------------------------------ standalone move
__global__ void __launch_bounds__(256)
k_apply(const float4 *__restrict__ st_in, const float4 *__restrict__ force, uint32_t n,
        ug_params P, float4 *st_out, float4 *disp_out, int32_t *status) {
    if (cta_failed(status)) return;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = st_in[i];
    const float4 F = force[i];
    bool moving;
    const float3 u = displacement(F.x, F.y, F.z, p.w, P, &moving);
    st_out[i] = make_float4(p.x + u.x, p.y + u.y, p.z + u.z, p.w);
    if (disp_out) disp_out[i] = make_float4(u.x, u.y, u.z, moving ? 1.f : 0.f);
}

void launch_apply(const float4 *st_in, const float4 *force, uint32_t n, const ug_params &p,
                  float4 *st_out, float4 *disp_out, int32_t *status, cudaStream_t s) {
    k_apply<<<(n + 255) / 256, 256, 0, s>>>(st_in, force, n, p, st_out, disp_out, status);
}

}  // namespace ug
