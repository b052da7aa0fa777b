// The paper's GPU version ladder (Hesam et al., Sec. IV-B to IV-E), rebuilt
// for comparison with the main path; never used by it.
//
//   version 0  one thread per agent walks the 27 boxes of a per-box linked list
//              (the uniform grid of Sec. IV-A: each box knows its last agent,
//              each agent the one added before it) over the rows in the
//              caller's order, Eq. 1 in float64
//   version 1  the same in float32 (Sec. IV-C)
//   version 2  the same over box-sorted rows (Sec. IV-D; the box order of the
//              main path's counting sort stands in for the Z-order curve)
//              (the linked lists hold one entry per box, whatever the number
//              of x sub-bins the main path's box table has per box)
//   version 3  one CTA per box: the agents of the 27 surrounding boxes are
//              appended to shared memory through an atomic counter, then the
//              box's agents are tested against that shared neighbourhood
//              (Sec. IV-E), float32, box-sorted rows
//
// All four evaluate Eq. 1 directly (delta = r_i + r_j + 2m - d, plain sums in
// the version's precision), with the grid geometry of the main path.  The
// linked lists are built with atomicExch, so their order, and with it the
// float32 sums of versions 1-3, may differ from run to run.
#include <cuda_runtime.h>

#include "ug_internal.cuh"

namespace ug {

constexpr uint32_t kNone = 0xffffffffu;
constexpr int kLadderShared = 1024;   // neighbourhood rows a version-3 CTA can hold

// Per-box linked lists: head[key] = last agent added, next[i] = the agent added
// before i (kNone ends a list).  head must hold kNone for every box on entry.
__global__ void __launch_bounds__(256)
k_ll_build(const float4 *__restrict__ rows, uint32_t n, const ug_grid_info *__restrict__ geo,
           uint32_t *head, uint32_t *__restrict__ next, int32_t *status) {
    if (cta_failed(status)) return;
    const ug_grid_info g = geo[0];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int bx, by, bz;
        box_key(__ldg(rows + i), g, bx, by, bz);
        const uint32_t k = (uint32_t)((bz * g.dims[1] + by) * g.dims[0] + bx);   // one list per box
        next[i] = atomicExch(&head[k], i);
    }
}

__device__ __forceinline__ float root_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double root_t(double x) { return sqrt(x); }

// Eq. 1 for agent a and neighbour b, written out directly in precision T;
// adds the force on a to (fx, fy, fz) and returns whether the pair overlaps.
template <typename T>
__device__ __forceinline__ bool eq1_direct(const float4 &a, const float4 &b, T m2, T k, T gamma,
                                           T &fx, T &fy, T &fz) {
    const T hx = (T)a.x - (T)b.x, hy = (T)a.y - (T)b.y, hz = (T)a.z - (T)b.z;
    const T d = root_t(hx * hx + hy * hy + hz * hz);
    const T ra = (T)0.5 * (T)a.w, rb = (T)0.5 * (T)b.w;
    const T delta = ra + rb + m2 - d;
    if (!(delta > (T)0) || !(d > (T)0)) return false;
    const T R = ra * rb / (ra + rb);
    const T c = (k * delta - gamma * root_t(R * delta)) / d;
    fx += c * hx;
    fy += c * hy;
    fz += c * hz;
    return true;
}

// Versions 0-2: one thread per agent over the 27 boxes' linked lists.  A list
// holds each agent once (atomicExch), so a walk ends after at most n links;
// the bound is checked anyway.
template <typename T>
__global__ void __launch_bounds__(128)
k_ll_force(const float4 *__restrict__ rows, uint32_t n, const ug_grid_info *__restrict__ geo,
           const uint32_t *__restrict__ head, const uint32_t *__restrict__ next, ug_params P,
           const uint32_t *__restrict__ ids, double *__restrict__ force, int32_t *status) {
    if (cta_failed(status)) return;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ug_grid_info g = geo[0];
    const float4 me = __ldg(rows + i);
    int bx, by, bz;
    box_key(me, g, bx, by, bz);
    const T m2 = (T)2 * (T)P.contact_margin, k = (T)P.k, gamma = (T)P.gamma;
    T fx = 0, fy = 0, fz = 0;
    uint32_t np = 0, links = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const uint32_t key =
                    (uint32_t)(((bz + dz) * g.dims[1] + (by + dy)) * g.dims[0] + (bx + dx));
                for (uint32_t j = __ldg(head + key); j != kNone; j = __ldg(next + j)) {
                    if (++links > n) { set_status(status, UG_EBADSTATE); return; }
                    if (j != i && eq1_direct<T>(me, __ldg(rows + j), m2, k, gamma, fx, fy, fz)) ++np;
                }
            }
    const uint32_t o = ids ? __ldg(ids + i) : i;
    force[4 * (size_t)o + 0] = (double)fx;
    force[4 * (size_t)o + 1] = (double)fy;
    force[4 * (size_t)o + 2] = (double)fz;
    force[4 * (size_t)o + 3] = (double)np;
}

// Version 3: CTAs of 32 threads take boxes in a grid stride.  Threads 0..26
// each append one neighbour box's agents (rows and sorted indices) to shared
// memory, taking slots from an atomic counter; then every thread takes agents
// of its box and tests them against all appended rows.
__global__ void __launch_bounds__(32)
k_box_shared(const float4 *__restrict__ rows, const uint32_t *__restrict__ start,
             const ug_grid_info *__restrict__ geo, const Ctrl *ctrl, ug_params P,
             const uint32_t *__restrict__ ids, double *__restrict__ force, int32_t *status) {
    __shared__ float4 s_rows[kLadderShared];
    __shared__ uint32_t s_idx[kLadderShared];
    __shared__ uint32_t s_cnt;
    if (cta_failed(status)) return;
    const ug_grid_info g = geo[0];
    // boxes of the grid (0 after a failed build); box b's rows are table
    // entries b K .. (b + 1) K, K = 2^ks x sub-bins per box
    const uint32_t total = *(volatile const uint32_t *)&ctrl->total_boxes ? g.nboxes : 0u;
    const int ks = grid_shift(g);
    const float m2 = 2.0f * P.contact_margin;
    const int t = threadIdx.x;
    for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
        const uint32_t a0 = __ldg(start + (b << ks)), a1 = __ldg(start + ((b + 1) << ks));
        if (a0 == a1) continue;   // CTA-uniform: only boxes with agents (always interior)
        if (t == 0) s_cnt = 0u;
        __syncthreads();
        if (t < 27) {
            const int off = (t / 9 - 1) * g.dims[0] * g.dims[1] + (t / 3 % 3 - 1) * g.dims[0] + (t % 3 - 1);
            const uint32_t kb = (uint32_t)((int)b + off);
            const uint32_t j0 = __ldg(start + (kb << ks)), j1 = __ldg(start + ((kb + 1) << ks));
            for (uint32_t j = j0; j < j1; ++j) {
                const uint32_t slot = atomicAdd(&s_cnt, 1u);
                if (slot < (uint32_t)kLadderShared) {
                    s_rows[slot] = __ldg(rows + j);
                    s_idx[slot] = j;
                }
            }
        }
        __syncthreads();
        const uint32_t cnt = s_cnt;
        if (cnt > (uint32_t)kLadderShared) {
            if (t == 0) set_status(status, UG_ECAPACITY);
        } else {
            for (uint32_t i = a0 + t; i < a1; i += 32) {
                const float4 me = __ldg(rows + i);
                float fx = 0.f, fy = 0.f, fz = 0.f;
                uint32_t np = 0;
                for (uint32_t s = 0; s < cnt; ++s)
                    if (s_idx[s] != i && eq1_direct<float>(me, s_rows[s], m2, P.k, P.gamma, fx, fy, fz)) ++np;
                const uint32_t o = __ldg(ids + i);
                force[4 * (size_t)o + 0] = (double)fx;
                force[4 * (size_t)o + 1] = (double)fy;
                force[4 * (size_t)o + 2] = (double)fz;
                force[4 * (size_t)o + 3] = (double)np;
            }
        }
        __syncthreads();
    }
}

int run_ladder(int version, const float4 *state, uint32_t n, const SimArgs &sa, uint32_t max_boxes,
               const Workspace &w, uint32_t *head, uint32_t *next, double *force, int32_t *status,
               cudaStream_t s) {
    launch_bounds(state, sa, w, w.geo, max_boxes, status, s);
    const unsigned tb = 128, nb = (unsigned)((n + tb - 1) / tb);
    const uint64_t bb_all = ((uint64_t)n + 255) / 256, bb_cap = 8ull * (uint64_t)device_sm_count();
    const unsigned bb = (unsigned)(bb_all < bb_cap ? bb_all : bb_cap);
    if (version <= 1) {
        if (cudaMemsetAsync(head, 0xff, sizeof(uint32_t) * (size_t)max_boxes, s) != cudaSuccess)
            return UG_ECUDA;
        k_ll_build<<<bb, 256, 0, s>>>(state, n, w.geo, head, next, status);
        if (version == 0)
            k_ll_force<double><<<nb, tb, 0, s>>>(state, n, w.geo, head, next, sa.pval, nullptr, force, status);
        else
            k_ll_force<float><<<nb, tb, 0, s>>>(state, n, w.geo, head, next, sa.pval, nullptr, force, status);
        return cudaGetLastError() == cudaSuccess ? UG_OK : UG_ECUDA;
    }
    // versions 2 and 3 work on box-sorted rows: the main path's grid build
    launch_key(state, sa, w, w.geo, nullptr, status, s);
    launch_scan(w, w.start, max_boxes, status, s);
    launch_place(w, w.start, n, status, s);
    launch_canon(w, w.start, state, nullptr, w.sorted, w.perm2, nullptr, n, status, s);
    if (version == 2) {
        if (cudaMemsetAsync(head, 0xff, sizeof(uint32_t) * (size_t)max_boxes, s) != cudaSuccess)
            return UG_ECUDA;
        k_ll_build<<<bb, 256, 0, s>>>(w.sorted, n, w.geo, head, next, status);
        k_ll_force<float><<<nb, tb, 0, s>>>(w.sorted, n, w.geo, head, next, sa.pval, w.perm2, force, status);
    } else {
        const uint64_t cap = 32ull * (uint64_t)device_sm_count();
        const unsigned grid = (unsigned)((uint64_t)max_boxes < cap ? (uint64_t)max_boxes : cap);
        k_box_shared<<<grid, 32, 0, s>>>(w.sorted, w.start, w.geo, w.ctrl, sa.pval, w.perm2, force, status);
    }
    return cudaGetLastError() == cudaSuccess ? UG_OK : UG_ECUDA;
}

}  // namespace ug
