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

template <int MODE, int T>
__global__ void __launch_bounds__(T)
k_sweep(const float4 *__restrict__ st, const uint32_t *__restrict__ start,
        const ug_grid_info *__restrict__ geo, const uint32_t *__restrict__ skey, SimArgs sa,
        SweepOut out, int32_t *status) {
    __shared__ uint32_t lst[kListCap][T];
    __shared__ uint2 runs[9][T];
    if (cta_failed(status)) return;
    const uint32_t first = blockIdx.x * T;
    const uint32_t i = first + threadIdx.x;
    const bool valid = i < sa.n;
    bool uniform;
    const uint32_t sim = cta_sim(sa, first, i, uniform);
    const ug_params P = sim_params(sa, sim);
    const ug_grid_info g = geo[sim];
    const float m2 = 2.0f * P.contact_margin;

    const float4 me = valid ? __ldg(st + i) : make_float4(0.f, 0.f, 0.f, 1.f);
    const float ri = 0.5f * me.w;
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    uint32_t np = 0;
    const uint32_t key_i = (skey != nullptr && valid) ? __ldg(skey + i) : 0xffffffffu;
    // filtered candidates lie within e (+ rounding) of row i: if every lane of
    // the warp is far from the coordinate planes their differences are exact
    const bool exact_diffs = __all_sync(kFull, !valid || far_from_origin(me, g.edge));
    sweep_neighbours<T>(st, start, g, i, valid, me, key_i, m2, runs, lst,
                        [&](uint32_t jj, const float4 &q) {
        ContactGeo c;
        const bool hit = exact_diffs ? contact_t<false>(me, ri, q, m2, c)
                                     : contact_t<true>(me, ri, q, m2, c);
        if (!hit) return;
        if (MODE == kSweepPairs) {
            if (np < out.max_per_agent) out.nbr[(size_t)i * out.max_per_agent + np] = jj;
        } else {
            const float R = __fdividef(ri * c.rb, c.rsum);
            const float rd = R * c.delta;
            const float root = rd * rsqrtf(rd);
            const float phi = P.k * c.delta - P.gamma * root;
            const float coef = phi * c.invd;
            comp_add(sx, cx, coef * c.hx);
            comp_add(sy, cy, coef * c.hy);
            comp_add(sz, cz, coef * c.hz);
        }
        ++np;
    });

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
    if (elect_last_cta(&out.ctrl->done))
        finalize_grid(sa, out.bounds, out.geo_next, out.ctrl, out.max_boxes, status);
}

template <int MODE>
static void launch_mode(const float4 *sorted, const uint32_t *start, const ug_grid_info *geo,
                        const SimArgs &sa, const SweepOut &out, int block, int32_t *status,
                        cudaStream_t s, const uint32_t *skey) {
    switch (block) {
    case 64:
        k_sweep<MODE, 64><<<(sa.n + 63) / 64, 64, 0, s>>>(sorted, start, geo, skey, sa, out, status);
        break;
    case 256:
        k_sweep<MODE, 256><<<(sa.n + 255) / 256, 256, 0, s>>>(sorted, start, geo, skey, sa, out,
                                                             status);
        break;
    default:
        k_sweep<MODE, 128><<<(sa.n + 127) / 128, 128, 0, s>>>(sorted, start, geo, skey, sa, out,
                                                             status);
        break;
    }
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
