// Reverse mode of the unrolled step: gradients of a loss on the final rows with
// respect to the initial rows (positions and diameters) and to Eq. 1's kappa
// and gamma.  The forward segment is recomputed from a checkpoint with every
// step's sorted rows, sort permutation, box table, geometry, forces and
// adherence/cap flags saved; the reverse sweep walks the same 27-box
// neighbourhoods on the saved grids.
//
// Per step t (rows in step t's box order, X_{t+1} = S_t + u(S_t)):
//   w_i   = dL/dX_{t+1}[i]
//   capped: w_i <- (max_disp/|v_i|)(I - v^ v^T) w_i,   v_i = dt/m_i F_i
//   g_i   = dt/m_i w_i if moving else 0          (= dL/dF_i)
//   dL/dd_i from the mass: -3 (w_i . v_i) / d_i if moving
//   for every contact (i, j), with u = (p_i - p_j)/d:
//     J_ij (g_i - g_j) = phi'(d) u (u.(g_i-g_j)) + phi/d ((g_i-g_j) - u (u.(g_i-g_j))),
//     phi'(d) = -(kappa - gamma R / (2 sqrt(R delta)))
//     dL/dkappa += (g_i . u) delta,  dL/dgamma -= (g_i . u) sqrt(R delta)
//     dL/dd_i   += (u.(g_i-g_j)) / 2 * dphi/dr_i,
//     dphi/dr_i = dphi/ddelta - gamma delta / (2 sqrt(R delta)) * r_j^2 / (r_i + r_j)^2
//   dL/dX_t[sigma_t[i]] = (w_i + sum_j J_ij (g_i - g_j), w_i.d + mass and contact terms)
// The adherence test, the cap branch and contact membership are piecewise
// constant and carry no derivative.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "ug_internal.cuh"

namespace ug {

constexpr int kAdjT = 128;

static inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct AdjLayout {
    Workspace fw;
    float4 *state;          // [n] working copy of the checkpoint
    uint32_t *perm;         // [n]
    StepSaves saves;
    float4 *G[2];           // [n] ping-pong adjoints of the rows
    float4 *g;              // [n] (g_i, mass part of dL/dd_i)
    float4 *partial;        // [nblk] float-float partial sums of dL/dkappa, dL/dgamma
    size_t bytes;
};

static size_t adj_layout(void *base, uint32_t n, uint32_t max_boxes, int nsteps, AdjLayout *L) {
    char *b = static_cast<char *>(base);
    size_t off = a256(layout_workspace(base, n, 1, max_boxes, &L->fw));
    auto take = [&](size_t bytes) -> char * {
        char *p = b ? b + off : nullptr;
        off = a256(off + bytes);
        return p;
    };
    const size_t S = (size_t)std::max(nsteps, 1);
    L->state = reinterpret_cast<float4 *>(take(16 * (size_t)n));
    L->perm = reinterpret_cast<uint32_t *>(take(4 * (size_t)n));
    L->saves.sorted = reinterpret_cast<float4 *>(take(16 * (size_t)n * S));
    L->saves.sigma = reinterpret_cast<uint32_t *>(take(4 * (size_t)n * S));
    L->saves.start_stride = ((size_t)table_capacity(n, max_boxes) + 1 + 63) & ~(size_t)63;
    L->saves.start = reinterpret_cast<uint32_t *>(take(4 * L->saves.start_stride * S));
    L->saves.force = reinterpret_cast<float4 *>(take(16 * (size_t)n * S));
    L->saves.geo = reinterpret_cast<ug_grid_info *>(take(sizeof(ug_grid_info) * S));
    L->G[0] = reinterpret_cast<float4 *>(take(16 * (size_t)n));
    L->G[1] = reinterpret_cast<float4 *>(take(16 * (size_t)n));
    L->g = reinterpret_cast<float4 *>(take(16 * (size_t)n));
    const size_t nblk = ((size_t)n + kAdjT - 1) / kAdjT;
    L->partial = reinterpret_cast<float4 *>(take(16 * std::max<size_t>(nblk, 1)));
    L->bytes = off;
    return off;
}

// ------------------------------------------------------------------ per-agent part
__global__ void __launch_bounds__(256)
k_adj_prep(const float4 *__restrict__ sorted, const float4 *__restrict__ force,
           const float4 *__restrict__ W, uint32_t n, ug_params P, float4 *__restrict__ g,
           int32_t *status) {
    if (cta_failed(status)) return;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 F = force[i];
    const int flags = (int)F.w;
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (flags & 1) {
        const float d = sorted[i].w;
        const float m = P.density * (float)(M_PI / 6.0) * d * d * d;
        const float c = P.dt / m;
        const float vx = c * F.x, vy = c * F.y, vz = c * F.z;
        const float4 Wi = W[i];
        float wx = Wi.x, wy = Wi.y, wz = Wi.z;
        if (flags & 2) {
            const float vn = sqrtf(vx * vx + vy * vy + vz * vz);
            const float ix = vx / vn, iy = vy / vn, iz = vz / vn;
            const float dot = ix * wx + iy * wy + iz * wz;
            const float sc = P.max_disp / vn;
            wx = sc * (wx - ix * dot);
            wy = sc * (wy - iy * dot);
            wz = sc * (wz - iz * dot);
        }
        out = make_float4(c * wx, c * wy, c * wz, -3.0f * (wx * vx + wy * vy + wz * vz) / d);
    }
    g[i] = out;
}

// ------------------------------------------------------------------ contact part
__global__ void __launch_bounds__(kAdjT)
k_adj_sweep(const float4 *__restrict__ st, const uint32_t *__restrict__ start,
            const ug_grid_info *__restrict__ geo, const float4 *__restrict__ g,
            const float4 *__restrict__ W, const uint32_t *__restrict__ sigma, uint32_t n,
            ug_params P, float4 *__restrict__ Gout, float4 *partial, int32_t *status) {
    __shared__ WarpLists wl[kAdjT / 32];
    __shared__ float s_red[2][kAdjT / 32];
    if (cta_failed(status)) return;
    const uint32_t i = blockIdx.x * kAdjT + threadIdx.x;
    const bool valid = i < n;
    const ug_grid_info gi_geo = geo[0];
    const float m2 = 2.0f * P.contact_margin;
    const float4 me = valid ? __ldg(st + i) : make_float4(0.f, 0.f, 0.f, 1.f);
    const float4 gi = valid ? __ldg(g + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float ri = 0.5f * me.w;
    float ax = 0.f, ay = 0.f, az = 0.f, ad = 0.f, pk = 0.f, pg = 0.f;
    sweep_neighbours(st, start, gi_geo, i, valid, me, 0xffffffffu, m2, wl[threadIdx.x >> 5],
                            [&](uint32_t jj, const float4 &q) {
        ContactGeo c;
        if (!contact(me, ri, q, m2, c)) return;
        const float4 gj = __ldg(g + jj);
        const float R = __fdividef(ri * c.rb, c.rsum);
        const float rd = R * c.delta;
        const float root = rd * rsqrtf(rd);
        const float phi = P.k * c.delta - P.gamma * root;
        const float ux = c.hx * c.invd, uy = c.hy * c.invd, uz = c.hz * c.invd;
        const float gx = gi.x - gj.x, gy = gi.y - gj.y, gz = gi.z - gj.z;
        const float ug = ux * gx + uy * gy + uz * gz;
        const float half_root_inv = __fdividef(0.5f, root);
        const float dphi_ddelta = P.k - P.gamma * R * half_root_inv;
        const float a = phi * c.invd;
        const float b = -dphi_ddelta * ug - a * ug;
        ax += a * gx + b * ux;
        ay += a * gy + b * uy;
        az += a * gz + b * uz;
        const float giu = gi.x * ux + gi.y * uy + gi.z * uz;
        pk += giu * c.delta;
        pg -= giu * root;
        const float dphi_dR = -P.gamma * c.delta * half_root_inv;
        const float rr = __fdividef(c.rb, c.rsum);
        ad += ug * 0.5f * (dphi_ddelta + dphi_dR * rr * rr);
    });
    if (valid) {
        const float4 Wi = W[i];
        Gout[sigma[i]] = make_float4(Wi.x + ax, Wi.y + ay, Wi.z + az, Wi.w + gi.w + ad);
    }
    // deterministic CTA reduction of the parameter terms, accumulated per CTA
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pk += __shfl_down_sync(kFull, pk, o);
        pg += __shfl_down_sync(kFull, pg, o);
    }
    if (lane == 0) { s_red[0][warp] = pk; s_red[1][warp] = pg; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float tk = 0.f, tg = 0.f;
        for (int w = 0; w < kAdjT / 32; ++w) { tk += s_red[0][w]; tg += s_red[1][w]; }
        float4 acc = partial[blockIdx.x];
        comp_add(acc.x, acc.y, tk);
        comp_add(acc.z, acc.w, tg);
        partial[blockIdx.x] = acc;
    }
}

__global__ void __launch_bounds__(256)
k_adj_reduce(const float4 *__restrict__ partial, uint32_t nblk, float *grad_params) {
    __shared__ float s[4][256];
    float kh = 0.f, kl = 0.f, gh = 0.f, gl = 0.f;
    for (uint32_t b = threadIdx.x; b < nblk; b += blockDim.x) {
        const float4 p = partial[b];
        comp_add(kh, kl, p.x);
        kl += p.y;
        comp_add(gh, gl, p.z);
        gl += p.w;
    }
    s[0][threadIdx.x] = kh; s[1][threadIdx.x] = kl;
    s[2][threadIdx.x] = gh; s[3][threadIdx.x] = gl;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, ac = 0.f, c = 0.f, cc = 0.f;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            comp_add(a, ac, s[0][t]);
            ac += s[1][t];
            comp_add(c, cc, s[2][t]);
            cc += s[3][t];
        }
        grad_params[0] = a + ac;
        grad_params[1] = c + cc;
    }
}

}  // namespace ug

using namespace ug;

extern "C" {

size_t ug_backward_workspace_bytes(uint32_t n, uint32_t max_boxes, int32_t nsteps) {
    AdjLayout L;
    return adj_layout(nullptr, n, max_boxes, nsteps, &L);
}

int ug_step_backward(const float *ckpt_state, uint32_t n, ug_params p, int32_t nsteps,
                     uint32_t max_boxes, const float *grad_out, float *grad_in, float *grad_params,
                     void *ws, size_t ws_bytes, int32_t *status, void *stream) {
    if (nsteps < 0 || n > kMaxAgents) return UG_EINVAL;
    if (!grad_params || !status) return UG_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0 || nsteps == 0) {
        if (cudaMemsetAsync(grad_params, 0, 2 * sizeof(float), s) != cudaSuccess) return UG_ECUDA;
        if (n && nsteps == 0) {
            if (!grad_in || !grad_out) return UG_EINVAL;
            if (cudaMemcpyAsync(grad_in, grad_out, 16 * (size_t)n, cudaMemcpyDeviceToDevice, s) !=
                cudaSuccess)
                return UG_ECUDA;
        }
        return UG_OK;
    }
    if (!ckpt_state || !grad_out || !grad_in || !ws || ((uintptr_t)ws & 255) ||
        ((uintptr_t)ckpt_state & 15) || ((uintptr_t)grad_out & 15) || ((uintptr_t)grad_in & 15) ||
        max_boxes < 27 || max_boxes > 0x7fffff00u || !(p.contact_margin >= 0.0f))
        return UG_EINVAL;
    AdjLayout L;
    if (adj_layout(ws, n, max_boxes, nsteps, &L) > ws_bytes) return UG_EWORKSPACE;
    const uint32_t nblk = (n + kAdjT - 1) / kAdjT;
    if (cudaMemcpyAsync(L.state, ckpt_state, 16 * (size_t)n, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return UG_ECUDA;
    if (cudaMemsetAsync(L.perm, 0, 4 * (size_t)n, s) != cudaSuccess) return UG_ECUDA;
    if (cudaMemsetAsync(L.partial, 0, 16 * (size_t)nblk, s) != cudaSuccess) return UG_ECUDA;
    SimArgs sa{};
    sa.nsims = 1;
    sa.n = n;
    sa.pval = p;
    sa.bounds_copies = kBoundsCopiesSingle;
    int rc = run_steps(L.state, L.perm, sa, nsteps, max_boxes, L.fw, 128, 2, &L.saves, status, s,
                       nullptr, windows_pay(n, max_boxes));
    if (rc != UG_OK) return rc;
    const float4 *W = reinterpret_cast<const float4 *>(grad_out);
    int nb = 0;
    for (int t = nsteps - 1; t >= 0; --t) {
        const float4 *sorted = L.saves.sorted + (size_t)t * n;
        const float4 *force = L.saves.force + (size_t)t * n;
        float4 *Gout = t == 0 ? reinterpret_cast<float4 *>(grad_in) : L.G[nb];
        k_adj_prep<<<(n + 255) / 256, 256, 0, s>>>(sorted, force, W, n, p, L.g, status);
        k_adj_sweep<<<nblk, kAdjT, 0, s>>>(sorted, L.saves.start + (size_t)t * L.saves.start_stride,
                                           L.saves.geo + t, L.g, W, L.saves.sigma + (size_t)t * n,
                                           n, p, Gout, L.partial, status);
        W = Gout;
        nb ^= 1;
    }
    k_adj_reduce<<<1, 256, 0, s>>>(L.partial, nblk, grad_params);
    return cudaGetLastError() == cudaSuccess ? UG_OK : UG_ECUDA;
}

}  // extern "C"
