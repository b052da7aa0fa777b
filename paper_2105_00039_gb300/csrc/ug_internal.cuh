// Internal declarations shared by the library's translation units.
// Device helpers are header-inline; host launchers are defined in the .cu files.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ugmech.h"

namespace ug {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kScanThreads = 512;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;   // boxes per scan tile (a power of 2)
constexpr int kScanTileShift = 13;
static_assert(kScanTile == 1 << kScanTileShift, "scan tile must be 2^kScanTileShift boxes");
// Row counts per scan tile, kept as kTileCopies partial sums per tile (copy c
// of tile t at tile_sum[(t * kTileCopies + c) * kTileSumStride], each on its own
// 128-byte line), so that the histogram's per-warp atomics spread over many
// L2 lines instead of queueing on one per tile.
constexpr uint32_t kTileSumStride = 32;
constexpr uint32_t kTileCopies = 8;
constexpr uint32_t kMaxAgents = 1u << 30;               // largest n any entry point accepts
constexpr int kBoundsWords = 8;                         // per simulation, see bounds_*()
constexpr int kBoundsCopiesSingle = 32;                 // spread atomics when nsims == 1

// Control words living in the workspace (zeroed at the start of every call).
struct Ctrl {
    uint32_t spare;
    uint32_t done;          // CTAs finished (last-CTA pattern of the bounds reduction)
    uint32_t total_boxes;   // box table entries of the current grid (all sims); 0 after an error
    uint32_t adj_done;      // last-CTA counter of the adjoint parameter reduction
    uint32_t pad[4];
};

// Which simulation owns which rows, and its constants.
struct SimArgs {
    const uint32_t *offset;   // [nsims + 1] device, or nullptr: one simulation over [0, n)
    const ug_params *pdev;    // [nsims] device, or nullptr: pval for all
    ug_params pval;
    uint32_t nsims;
    uint32_t n;
    uint32_t bounds_copies;   // copies of the bounds accumulators (atomic spreading)
    bool per_box_table;       // the box table has one entry per box (a caller's table from
                              // ug_grid_build): kernels then ignore the geometry's sub-bins
};


// A simulation's geometry as a kernel uses it (see SimArgs::per_box_table).
__device__ __forceinline__ ug_grid_info sim_geo(const SimArgs &sa, const ug_grid_info *geo,
                                                uint32_t s) {
    ug_grid_info g = geo[s];
    if (sa.per_box_table) g.reserved = 0u;
    return g;
}

// ------------------------------------------------------------------ dependent launch
// Kernels of one step form a chain on the caller's stream.  Each is launched
// with programmatic stream serialization (launch_chained): it may be scheduled
// while its predecessor's last wave still runs, and waits at chain_begin() until
// the predecessor has completed and its writes are visible.  chain_begin() must
// be the first thing a chained kernel does.
__device__ __forceinline__ void chain_begin() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_chained(void (*kernel)(KArgs...), unsigned grid, unsigned block,
                           cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ------------------------------------------------------------------ status
__device__ __forceinline__ void set_status(int32_t *status, int32_t code) {
    atomicCAS(status, 0, code);
}
__device__ __forceinline__ int32_t peek_status(const int32_t *status) {
    return *(volatile const int32_t *)status;
}
// Block-uniform early exit: every thread of the CTA must call it.
__device__ __forceinline__ bool cta_failed(const int32_t *status) {
    __shared__ int s_fail;
    if (threadIdx.x == 0) s_fail = peek_status(status) != 0;
    __syncthreads();
    return s_fail != 0;
}

// ------------------------------------------------------------------ simulations
__device__ __forceinline__ uint32_t find_sim(const SimArgs &sa, uint32_t i) {
    if (sa.offset == nullptr || sa.nsims <= 1) return 0;
    uint32_t lo = 0, hi = sa.nsims;   // offset[lo] <= i < offset[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(sa.offset + mid) <= i) lo = mid; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ uint32_t sim_begin(const SimArgs &sa, uint32_t s) {
    return sa.offset ? __ldg(sa.offset + s) : 0u;
}
__device__ __forceinline__ uint32_t sim_end(const SimArgs &sa, uint32_t s) {
    return sa.offset ? __ldg(sa.offset + s + 1) : sa.n;
}
__device__ __forceinline__ ug_params sim_params(const SimArgs &sa, uint32_t s) {
    return sa.pdev ? sa.pdev[s] : sa.pval;
}
// Simulation of row i, resolved once per CTA when the CTA's rows share one.
// Every thread must call it.  `uniform` tells whether they do.
__device__ __forceinline__ uint32_t cta_sim(const SimArgs &sa, uint32_t first, uint32_t i,
                                            bool &uniform) {
    __shared__ uint32_t s_sim[2];
    if (sa.offset == nullptr || sa.nsims <= 1) { uniform = true; return 0; }
    if (threadIdx.x == 0) {
        const uint32_t last = min(first + blockDim.x, sa.n) - 1;
        s_sim[0] = find_sim(sa, min(first, sa.n - 1));
        s_sim[1] = find_sim(sa, last);
    }
    __syncthreads();
    uniform = s_sim[0] == s_sim[1];
    return uniform ? s_sim[0] : find_sim(sa, min(i, sa.n - 1));
}

// Simulation shared by the `count` rows from `first` (when they share one):
// every thread must call it; `uniform` tells whether they do.
__device__ __forceinline__ uint32_t cta_sim_range(const SimArgs &sa, uint32_t first,
                                                  uint32_t count, bool &uniform) {
    __shared__ uint32_t s_sr[2];
    if (sa.offset == nullptr || sa.nsims <= 1) { uniform = true; return 0; }
    if (threadIdx.x == 0) {
        s_sr[0] = find_sim(sa, min(first, sa.n - 1));
        s_sr[1] = find_sim(sa, min(first + count, sa.n) - 1);
    }
    __syncthreads();
    uniform = s_sr[0] == s_sr[1];
    return s_sr[0];
}

// ------------------------------------------------------------------ ordered floats
// Monotone map float -> uint32 (larger float, larger code); 0 is below every
// float, so a zeroed word is the identity of atomicMax.
__device__ __forceinline__ uint32_t ord_enc(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_dec(uint32_t e) {
    return __uint_as_float((e & 0x80000000u) ? (e & 0x7fffffffu) : ~e);
}

// ------------------------------------------------------------------ grid geometry
// Box coordinate along one axis: max(floor(t), 1) with t = (p - o) / e in IEEE
// float32 round-to-nearest subtraction and division (the oracle evaluates the
// same expression in float32).  The upper clamp never binds for rows the
// geometry was built from.  *t_out gets t itself (the position in box units).
__device__ __forceinline__ int box_coord(float p, float o, float e, int dim, float *t_out = nullptr) {
    const float t = __fdiv_rn(__fsub_rn(p, o), e);
    int b = (int)floorf(t);
    b = max(b, 1);
    b = min(b, dim - 2);
    if (t_out) *t_out = t;
    return b;
}

// Agents are ordered by box and, inside a box, by x sub-bin: the box edge is
// cut into K = 2^ks equal slices along x (sub-bin sx = floor((t_x - b_x) K),
// clamped into [0, K)), so that the three boxes of a neighbour row, walked in
// table order, are sorted by x at the resolution e / K and an agent's
// candidates in that row form a short window (the grid's purpose in Sec. IV-A
// and IV-D is locality; the finer x order is how this library serves it).
// K follows the simulation's density: the largest 2^ks <= 8 with
// 4 * K * boxes <= 5 * agents (about one agent per sub-bin or more), so K = 1
// for sparse grids.  The box table then holds K entries per box: entry
// box_base + (box << ks) + sx starts sub-bin sx of the box, and the K entries of a
// simulation's boxes add up to at most boxes + 1.25 agents.
constexpr int kSubShiftMax = 3;
__host__ __device__ __forceinline__ int sub_shift(uint32_t agents, unsigned long long boxes) {
    int ks = 0;
    while (ks < kSubShiftMax && 4ull * (boxes << (ks + 1)) <= 5ull * agents) ++ks;
    return boxes == 0 ? 0 : ks;
}
// Entries of a box table serving n agents in grids of at most max_boxes boxes.
__host__ __device__ __forceinline__ unsigned long long table_capacity(uint32_t n, uint32_t max_boxes) {
    return (unsigned long long)max_boxes + n + (n >> 2) + 1;
}
// Neighbour-row windows pay where candidates dominate.  Measured on GB300
// (4,194,304 cells): the windowed walk is 9% slower than the full runs at 8
// neighbours per agent and 6% slower at 2, and 13% / 15% faster at 32 / 64.
// The host cannot see a step's grid (it is built on the device), so it judges
// from the agents and the box capacity: max_boxes bounds the boxes from above,
// so the agents per box it sees never exceed the grid's.  Windows are used
// from 2 agents per box (measured on the 4M-cell density cube: equal to the
// full runs at 5 neighbours, 1.7 agents per box; 1.5% faster at 6, 2.1 agents
// per box; 3% at 7, 5% at 8, 10% at 10, 23-26% at 32-64).  Either walk gives
// the same bits, so a wrong guess costs time only.
inline bool windows_pay(uint32_t n, uint32_t max_boxes) {
    return (unsigned long long)n >= 2ull * max_boxes;
}
// The same judgement for the every-pair-once walk, whose forward half-rows are
// shorter and whose flush is cheaper, so the windows' set-up weighs more: from 8
// agents per box (measured on the same cube: 2% slower at 8 neighbours, 2.8
// agents per box; equal at 16; 2% faster at 32 and 6% at 64).
inline bool windows_pay_pairs_once(uint32_t n, uint32_t max_boxes) {
    return (unsigned long long)n >= 8ull * max_boxes;
}
__device__ __forceinline__ int grid_shift(const ug_grid_info &g) { return (int)g.reserved; }

// Table entry of the first sub-bin of the agent's box (the box key); bx, by, bz
// get the box coordinates.
__device__ __forceinline__ uint32_t box_key(const float4 &p, const ug_grid_info &g,
                                            int &bx, int &by, int &bz) {
    bx = box_coord(p.x, g.origin[0], g.edge, g.dims[0]);
    by = box_coord(p.y, g.origin[1], g.edge, g.dims[1]);
    bz = box_coord(p.z, g.origin[2], g.edge, g.dims[2]);
    return g.box_base + ((uint32_t)((bz * g.dims[1] + by) * g.dims[0] + bx) << grid_shift(g));
}
// Sort key of an agent: its box key plus its x sub-bin.
__device__ __forceinline__ uint32_t sort_key(const float4 &p, const ug_grid_info &g) {
    float tx;
    const int bx = box_coord(p.x, g.origin[0], g.edge, g.dims[0], &tx);
    const int by = box_coord(p.y, g.origin[1], g.edge, g.dims[1]);
    const int bz = box_coord(p.z, g.origin[2], g.edge, g.dims[2]);
    const int ks = grid_shift(g);
    const int K = 1 << ks;
    // t_x - b_x is exact (Sterbenz) and scaling by K is exact
    int sx = (int)floorf(__fmul_rn(__fsub_rn(tx, (float)bx), (float)K));
    sx = min(max(sx, 0), K - 1);
    return g.box_base + ((uint32_t)((bz * g.dims[1] + by) * g.dims[0] + bx) << ks) + (uint32_t)sx;
}
// The box key of a sort key.
__device__ __forceinline__ uint32_t box_of_sort_key(uint32_t k, const ug_grid_info &g) {
    return k - ((k - g.box_base) & ((1u << grid_shift(g)) - 1u));
}

// ------------------------------------------------------------------ neighbour-row windows
// With K = 2^ks table entries per box (x sub-bins, see sort_key) the three boxes
// of a neighbour row are sorted by x at resolution e / K.  An agent's contacts
// in row (dy, dz) lie within
//   |x_j - x_i| < w,  w^2 = S_i^2 - g_y^2 - g_z^2,
// where S_i >= r_i + r_j + 2m for every j (r_i + m + e / 2, as e >= d_max + 2m)
// and g_y, g_z are the distances from the agent to that row's faces (0 for its
// own row or plane), so the row's candidates are the sub-bins overlapping
// [x_i - w, x_i + w]: two table reads give the window.  Everything is done in
// box units, t = (p - o) / e exactly as the sort computes it, with slack for
// its rounding (t carries at most 2^-23 relative error, so every window is
// widened by (dims + 2) 2^-20 box units and the gaps narrowed by as much) and
// S_i inflated by 2^-14, so no contact is ever outside its window.  A row with
// w^2 <= 0 holds no candidate.  Contacts are met in the same order as over the
// full runs (rows by (dz, dy), ascending slots), so the sums are the same bits.
// The two-agent sweep (k_sweep2) and the every-pair-once walk (k_sym) use them.
constexpr float kWinInflate = 1.0f + 1.0f / 16384.0f;   // on S_i / e
constexpr float kWinRootInflate = 1.0f + 1.0f / 1048576.0f;   // on the approximate root
constexpr float kWinSlack = 1.0f / 1048576.0f;           // box units per box of extent

// An agent's place in the grid, in box units.
struct AgentBox {
    float tx, fy, fz;   // x position; fractional y and z positions in the box
    float su;           // largest contact distance / e, inflated
    int bx, by, bz;
};
__device__ __forceinline__ AgentBox agent_box(const float4 &p, const ug_grid_info &g, float inv_e,
                                              float m) {
    AgentBox a;
    float ty, tz;
    a.bx = box_coord(p.x, g.origin[0], g.edge, g.dims[0], &a.tx);
    a.by = box_coord(p.y, g.origin[1], g.edge, g.dims[1], &ty);
    a.bz = box_coord(p.z, g.origin[2], g.edge, g.dims[2], &tz);
    a.fy = fminf(fmaxf(__fsub_rn(ty, (float)a.by), 0.0f), 1.0f);   // exact for rows of the grid
    a.fz = fminf(fmaxf(__fsub_rn(tz, (float)a.bz), 0.0f), 1.0f);
    a.su = (0.5f + (0.5f * p.w + m) * inv_e) * kWinInflate;
    return a;
}

// Sub-bins [lo, hi] along the row (dy, dz) of the agent's box that can hold
// its contacts; false when none can.
__device__ __forceinline__ bool row_window(const AgentBox &a, int dy, int dz, float sly, float slz,
                                           float slx, float Kf, int K, int &lo, int &hi) {
    const float gy = dy == 0 ? 0.0f : fmaxf((dy < 0 ? a.fy : 1.0f - a.fy) - sly, 0.0f);
    const float gz = dz == 0 ? 0.0f : fmaxf((dz < 0 ? a.fz : 1.0f - a.fz) - slz, 0.0f);
    const float w2 = a.su * a.su - gy * gy - gz * gz;
    if (!(w2 > 0.0f)) return false;
    const float wx = w2 * rsqrtf(w2) * kWinRootInflate + slx;
    lo = max((int)floorf((a.tx - wx) * Kf), (a.bx - 1) * K);
    hi = min((int)floorf((a.tx + wx) * Kf), (a.bx + 1) * K + K - 1);
    return lo <= hi;
}

// ------------------------------------------------------------------ float-float
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
// Compensated accumulation (Knuth TwoSum, Neumaier-style running error).
__device__ __forceinline__ void comp_add(float &s, float &c, float x) {
    float t, e;
    two_sum(s, x, t, e);
    s = t;
    c = __fadd_rn(c, e);
}

// Contact test of Eq. 1 in float-float arithmetic.
//   a, b: rows (x, y, z, d); ra = a.w / 2; m2 = 2 * contact margin.
// q = s^2 - d^2 with s = ra + rb + m2 is formed from exact differences, exact
// squares and TwoSums, so its sign (the predicate delta > 0) and value are exact
// to ~1e-12 of s^2; delta = q / (s + d) then carries ~3 ulp of relative error.
// Returns false for no contact or coincident centres (d = 0).
struct ContactGeo {
    float delta;   // overlap
    float invd;    // 1 / |p_a - p_b|
    float hx, hy, hz;   // p_a - p_b (rounded)
    float rb;      // radius of b
    float rsum;    // ra + rb (rounded)
};
// Eq. 1 for one contact: the force on a from b is coef * (p_a - p_b) with
// coef = (kappa delta - gamma sqrt(R delta)) / d.  Returns coef; *root_out gets
// sqrt(R delta).  Explicit roundings keep it bit-identical across kernels.
__device__ __forceinline__ float eq1_coef(float ra, float rb, float rsum, float delta, float invd,
                                          float k, float gamma, float *root_out = nullptr) {
    const float R = __fdividef(__fmul_rn(ra, rb), rsum);
    const float rd = __fmul_rn(R, delta);
    const float root = __fmul_rn(rd, rsqrtf(rd));
    if (root_out) *root_out = root;
    const float phi = __fmaf_rn(k, delta, -__fmul_rn(gamma, root));
    return __fmul_rn(phi, invd);
}

// EXACT_DIFF = false assumes p_a - p_b is exact in float32, which holds by
// Sterbenz's lemma when |coordinate of a| >= 3 e on every axis and |p_a - p_b|
// is below the box edge e (see far_from_origin); the residual terms are then 0.
template <bool EXACT_DIFF>
__device__ __forceinline__ bool contact_t(const float4 &a, float ra, const float4 &b, float m2,
                                          ContactGeo &c) {
    float lx = 0.f, ly = 0.f, lz = 0.f;
    if (EXACT_DIFF) {
        two_sum(a.x, -b.x, c.hx, lx);
        two_sum(a.y, -b.y, c.hy, ly);
        two_sum(a.z, -b.z, c.hz, lz);
    } else {
        c.hx = __fsub_rn(a.x, b.x);
        c.hy = __fsub_rn(a.y, b.y);
        c.hz = __fsub_rn(a.z, b.z);
    }
    float px, ex, py, ey, pz, ez;
    two_prod(c.hx, c.hx, px, ex);
    two_prod(c.hy, c.hy, py, ey);
    two_prod(c.hz, c.hz, pz, ez);
    float s1, e1, D, e2;
    two_sum(px, py, s1, e1);
    two_sum(s1, pz, D, e2);
    // every rounding below is spelled out (no compiler FMA contraction), so the
    // result is the same bits in every kernel that inlines this
    float E = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(ex, ey), ez), e1), e2);
    if (EXACT_DIFF)
        E = __fmaf_rn(2.0f, __fmaf_rn(c.hx, lx, __fmaf_rn(c.hy, ly, __fmul_rn(c.hz, lz))), E);
    c.rb = 0.5f * b.w;
    float sh, sl;
    two_sum(ra, c.rb, sh, sl);
    c.rsum = sh;
    if (m2 != 0.0f) {
        float t, te;
        two_sum(sh, m2, t, te);
        sh = t;
        sl = __fadd_rn(sl, te);
    }
    float S2, S2e;
    two_prod(sh, sh, S2, S2e);
    S2e = __fmaf_rn(__fmul_rn(2.0f, sh), sl, S2e);
    const float q = __fadd_rn(__fsub_rn(S2, D), __fsub_rn(S2e, E));
    if (!(q > 0.0f) || !(D > 0.0f)) return false;
    c.invd = rsqrtf(D);
    const float d = __fmul_rn(D, c.invd);
    c.delta = __fdividef(q, __fadd_rn(sh, d));
    return true;
}
__device__ __forceinline__ bool contact(const float4 &a, float ra, const float4 &b, float m2,
                                        ContactGeo &c) {
    return contact_t<true>(a, ra, b, m2, c);
}
// True when every float32 difference p_a - p_b with |p_a - p_b| < e is exact.
__device__ __forceinline__ bool far_from_origin(const float4 &a, float e) {
    const float lim = 3.0f * e;
    return fabsf(a.x) >= lim && fabsf(a.y) >= lim && fabsf(a.z) >= lim;
}

// ------------------------------------------------------------------ FP32x2 pairs
// The exact contact test and Eq. 1 of two pairs at once, in Blackwell's FP32x2
// instructions (the two-agent sweep: entry k of each of the lane's two agents'
// lists).  Every packed
// operation rounds each half as the scalar one does, and the sequence is
// contact_t's and eq1_coef's, so the results are the same bits (the two-agent
// sweep is tested against the batched sweep's scalar flush).  Two rules keep it
// so: the compiler may fuse a packed multiply into a packed add that consumes
// it, so every rounded product that feeds an add or a subtraction is formed with
// scalar __fmul_rn (never fused); and where a half holds no candidate, or no
// contact, the two-agent sweep adds an exact zero (cz = 0), which leaves a
// compensated sum and its error term unchanged (a running sum that starts at +0
// never becomes -0).
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a product that an add or a subtraction consumes (see above)
__device__ __forceinline__ float2 mul2_unfused(float2 a, float2 b) {
    return pk(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
}
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
    s = add2(a, b);
    const float2 bp = sub2(s, a);
    const float2 ap = sub2(s, bp);
    e = add2(sub2(a, ap), sub2(b, bp));
}
__device__ __forceinline__ void two_prod2(float2 a, float2 b, float2 &p, float2 &e) {
    p = mul2_unfused(a, b);
    e = fma2(a, b, neg2(p));
}

// The exact contact test (contact_t) and Eq. 1 (eq1_coef) of two pairs at once,
// (a0, b0) and (a1, b1), as the two halves of FP32x2 operations, bit for bit as
// the scalar functions compute them.  a* are given as packed x, y, z and radius;
// h0, h1 say which halves hold a listed candidate.  Returns the contact flags
// and, for contacts, the force coefficient (coef * (p_a - p_b) is the force on
// a) and p_a - p_b.  DIFFS_EXACT: the float32 centre differences are exact
// (far_from_origin), else they are formed with TwoSum.
template <bool DIFFS_EXACT>
__device__ __forceinline__ void contact_eq1_x2(float2 ax, float2 ay, float2 az, float2 ra,
                                               const float4 &q0, const float4 &q1, bool h0, bool h1,
                                               float m2, float2 kk, float2 gg, float2 &hx,
                                               float2 &hy, float2 &hz, float2 &coef, bool &t0,
                                               bool &t1) {
    const float2 bx = pk(q0.x, q1.x), by = pk(q0.y, q1.y), bz = pk(q0.z, q1.z);
    float2 lx = pk(0.f, 0.f), ly = pk(0.f, 0.f), lz = pk(0.f, 0.f);
    if (DIFFS_EXACT) {
        hx = sub2(ax, bx);
        hy = sub2(ay, by);
        hz = sub2(az, bz);
    } else {
        two_sum2(ax, neg2(bx), hx, lx);
        two_sum2(ay, neg2(by), hy, ly);
        two_sum2(az, neg2(bz), hz, lz);
    }
    float2 px, ex, py, ey, pz, ez;
    two_prod2(hx, hx, px, ex);
    two_prod2(hy, hy, py, ey);
    two_prod2(hz, hz, pz, ez);
    float2 s1, e1, D, e2;
    two_sum2(px, py, s1, e1);
    two_sum2(s1, pz, D, e2);
    float2 E = add2(add2(add2(add2(ex, ey), ez), e1), e2);
    if (!DIFFS_EXACT)
        E = fma2(pk(2.0f, 2.0f), fma2(hx, lx, fma2(hy, ly, mul2(hz, lz))), E);
    const float2 rb = mul2(pk(0.5f, 0.5f), pk(q0.w, q1.w));   // exact
    float2 sh, sl;
    two_sum2(ra, rb, sh, sl);
    const float2 rsum = sh;
    if (m2 != 0.0f) {
        float2 t, te;
        two_sum2(sh, pk(m2, m2), t, te);
        sh = t;
        sl = add2(sl, te);
    }
    float2 S2, S2e;
    two_prod2(sh, sh, S2, S2e);
    S2e = fma2(mul2(pk(2.0f, 2.0f), sh), sl, S2e);            // 2 sh: exact
    const float2 q = add2(sub2(S2, D), sub2(S2e, E));
    t0 = h0 && q.x > 0.0f && D.x > 0.0f;
    t1 = h1 && q.y > 0.0f && D.y > 0.0f;
    const float2 invd = pk(rsqrtf(D.x), rsqrtf(D.y));
    const float2 den = add2(sh, mul2_unfused(D, invd));
    const float2 delta = pk(__fdividef(q.x, den.x), __fdividef(q.y, den.y));
    const float2 rr = mul2(ra, rb);
    const float2 R = pk(__fdividef(rr.x, rsum.x), __fdividef(rr.y, rsum.y));
    const float2 rd = mul2(R, delta);
    const float2 root = pk(__fmul_rn(rd.x, rsqrtf(rd.x)), __fmul_rn(rd.y, rsqrtf(rd.y)));
    const float2 phi = fma2(kk, delta, neg2(mul2(gg, root)));
    coef = mul2(phi, invd);
}

// ------------------------------------------------------------------ neighbour traversal
// With boxes numbered x-fastest the 27 boxes around box key k are 9 runs of 3
// consecutive boxes, one per (dy, dz): with K table entries per box, row
// stride R = K dims_x and plane stride K dims_x dims_y, run (dy, dz) covers
// sorted slots start[k + dz*plane + dy*R - K] .. start[k + dz*plane + dy*R + 2K].
constexpr int kListCap = 20;
// The filter's relative band on the squared contact distance: the distance s
// is scaled by c = 1 + 2^-17 (exact in float32, c^2 > 1 + 2^-16), so the
// band costs no instruction per candidate.  The float32 roundings of d^2 and
// (c s)^2 stay below 2^-21 relative, far inside it: every pair with
// d < s passes.
constexpr float kFilterRoot = 1.0f + 1.0f / 131072.0f;

// The float32 pre-filter of one candidate row q against row i, in Blackwell's
// packed FP32x2 arithmetic: (dx, dy) = q.xy - p_i.xy and (dz, c s) =
// (q.z, q.w) * (1, c/2) + (-z_i, c (r_i + 2m)) are one instruction each, the
// squares two more.  True when |p_i - q|^2 < c^2 (r_i + r_q + 2m)^2, up to
// rounding.
struct FilterRow {
    float2 nxy;   // (-x_i, -y_i)
    float2 zr;    // (-z_i, c (r_i + 2m))
};
__device__ __forceinline__ FilterRow make_filter_row(const float4 &me, float m2) {
    FilterRow f;
    f.nxy = make_float2(-me.x, -me.y);
    f.zr = make_float2(-me.z, (0.5f * me.w + m2) * kFilterRoot);
    return f;
}
__device__ __forceinline__ bool prefilter(const float4 &q, const FilterRow &f) {
    const float2 dxy = __fadd2_rn(make_float2(q.x, q.y), f.nxy);
    const float2 dzs = __ffma2_rn(make_float2(q.z, q.w), make_float2(1.0f, 0.5f * kFilterRoot), f.zr);
    const float2 sxy = __fmul2_rn(dxy, dxy);
    const float2 szs = __fmul2_rn(dzs, dzs);
    const float d2 = sxy.x + sxy.y + szs.x;
    return d2 < szs.y;
}

// Visit every candidate j != i of the 27 boxes around row i; `fn(j, row_j)` is
// called for those passing a float32 distance filter whose 2^-16 relative band
// keeps every true contact (the exact test is fn's job).
//   key_i   the row's box key (box_key), or 0xffffffff to compute it from the position
//   w       this warp's candidate lists
// The 9 runs are visited one after another; inside a run every lane tests its
// t-th candidate in lockstep (trip count = the warp's longest run), with the
// index clamped into the lane's run and the result masked, so the loop body
// has no divergent branch.  Candidates passing the filter are handed to fn in
// warp-converged batches so that the exact, expensive path never runs one lane
// at a time.  All 32 lanes of every warp must call this.
constexpr int kSweepUnroll = 4;

struct WarpLists {            // per-warp scratch of sweep_neighbours (shared memory)
    uint32_t lst[kListCap][32];
};

template <typename Fn>
__device__ __forceinline__ void sweep_neighbours(const float4 *__restrict__ st,
                                                 const uint32_t *__restrict__ start,
                                                 const ug_grid_info &g, uint32_t i, bool valid,
                                                 const float4 &me, uint32_t key_i, float m2,
                                                 WarpLists &w, Fn &&fn) {
    const int lane = threadIdx.x & 31;
    uint32_t key = 0;
    if (valid) {
        key = key_i;
        if (key == 0xffffffffu) {
            int bx, by, bz;
            key = box_key(me, g, bx, by, bz);
        }
    }
    const int ks = grid_shift(g);
    const int row = g.dims[0] << ks, plane = (g.dims[0] * g.dims[1]) << ks;
    const uint32_t K = 1u << ks;
    const uint32_t self = valid ? i : 0u;
    const FilterRow fr = make_filter_row(me, m2);
    int cnt = 0;
    auto flush = [&]() {
        const int m = (int)__reduce_max_sync(kFull, (unsigned)cnt);
        for (int k = 0; k < m; ++k) {
            if (k < cnt) {
                const uint32_t jj = w.lst[k][lane];
                fn(jj, __ldg(st + jj));
            }
        }
        cnt = 0;
    };
#pragma unroll 1
    for (int r = 0; r < 9; ++r) {
        uint32_t b = self;
        int len = 0;
        if (valid) {
            const uint32_t kb = (uint32_t)((int)key + (r / 3 - 1) * plane + (r % 3 - 1) * row);
            b = __ldg(start + kb - K);
            len = (int)(__ldg(start + kb + 2 * K) - b);
            if (len == 0) b = self;
        }
        const int last = max(len - 1, 0);
        const int lmax = (int)__reduce_max_sync(kFull, (unsigned)len);
        for (int t = 0; t < lmax; t += kSweepUnroll) {
#pragma unroll
            for (int u = 0; u < kSweepUnroll; ++u) {
                const uint32_t jc = b + (uint32_t)min(t + u, last);
                const float4 cur = __ldg(st + jc);
                if ((t + u < len) & (jc != self) & prefilter(cur, fr)) {
                    w.lst[cnt][lane] = jc;
                    ++cnt;
                }
            }
            if (__any_sync(kFull, cnt > kListCap - kSweepUnroll)) flush();
        }
    }
    flush();
}

// ------------------------------------------------------------------ displacement
// Sec. III readings: moving iff |F| > adherence; v = dt/m F, m = rho pi/6 d^3;
// |v| capped at max_disp.  Returns u; *moving and *vn for the adjoint.
__device__ __forceinline__ float3 displacement(float Fx, float Fy, float Fz, float diam,
                                               const ug_params &P, bool *moving_out = nullptr,
                                               bool *capped_out = nullptr) {
    const float Fn = __fsqrt_rn(__fmaf_rn(Fx, Fx, __fmaf_rn(Fy, Fy, __fmul_rn(Fz, Fz))));
    float3 u = make_float3(0.f, 0.f, 0.f);
    bool moving = Fn > P.adherence, capped = false;
    if (moving) {
        const float m = __fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(P.density, (float)(M_PI / 6.0)),
                                                      diam), diam), diam);
        const float c = __fdiv_rn(P.dt, m);
        u = make_float3(__fmul_rn(c, Fx), __fmul_rn(c, Fy), __fmul_rn(c, Fz));
        const float vn = __fsqrt_rn(__fmaf_rn(u.x, u.x, __fmaf_rn(u.y, u.y, __fmul_rn(u.z, u.z))));
        if (vn > P.max_disp) {
            const float s = __fdiv_rn(P.max_disp, vn);
            u = make_float3(__fmul_rn(u.x, s), __fmul_rn(u.y, s), __fmul_rn(u.z, s));
            capped = true;
        }
    }
    if (moving_out) *moving_out = moving;
    if (capped_out) *capped_out = capped;
    return u;
}

// ------------------------------------------------------------------ bounds
// Per simulation and copy, kBoundsWords ordered codes maximised with atomicMax:
//   0..2 -min(x,y,z)   3..5 max(x,y,z)   6 max diameter   7 -min diameter
__device__ __forceinline__ void bounds_codes(const float4 &p, bool valid, uint32_t v[8]) {
    v[0] = valid ? ord_enc(-p.x) : 0u;
    v[1] = valid ? ord_enc(-p.y) : 0u;
    v[2] = valid ? ord_enc(-p.z) : 0u;
    v[3] = valid ? ord_enc(p.x) : 0u;
    v[4] = valid ? ord_enc(p.y) : 0u;
    v[5] = valid ? ord_enc(p.z) : 0u;
    v[6] = valid ? ord_enc(p.w) : 0u;
    v[7] = valid ? ord_enc(-p.w) : 0u;
}
__device__ __forceinline__ bool row_ok(const float4 &p) {
    return isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w) && p.w > 0.0f;
}

// Accumulate per-thread bounds codes (see bounds_codes; 0 = nothing); every
// thread of the CTA calls it.  `red` is shared-memory scratch: warp w uses the
// 8 words at red + w * red_stride (a kernel may point them into memory its
// warps no longer need, each warp into its own part).
__device__ __forceinline__ void accumulate_bounds_codes(const SimArgs &sa, uint32_t v[8],
                                                        bool valid, uint32_t sim, bool uniform,
                                                        uint32_t *bounds, uint32_t *red,
                                                        uint32_t red_stride) {
    const uint32_t copy = sa.bounds_copies > 1 ? blockIdx.x % sa.bounds_copies : 0u;
    if (uniform) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = __reduce_max_sync(kFull, v[k]);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 8; ++k) red[warp * red_stride + k] = v[k];
        }
        __syncthreads();
        if (threadIdx.x < 8) {
            uint32_t m = 0;
            const int nw = (blockDim.x + 31) >> 5;
            for (int w = 0; w < nw; ++w) m = max(m, red[w * red_stride + threadIdx.x]);
            if (m) atomicMax(&bounds[((size_t)copy * sa.nsims + sim) * kBoundsWords + threadIdx.x], m);
        }
    } else if (valid) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            atomicMax(&bounds[((size_t)copy * sa.nsims + sim) * kBoundsWords + k], v[k]);
    }
}

// Accumulate the bounds of one row per thread; every thread of the CTA calls it.
__device__ __forceinline__ void accumulate_bounds(const SimArgs &sa, const float4 &p, bool valid,
                                                  uint32_t sim, bool uniform, uint32_t *bounds,
                                                  int32_t *status) {
    __shared__ uint32_t s_red[32 * kBoundsWords];
    if (valid && !row_ok(p)) set_status(status, UG_EBADSTATE);
    uint32_t v[8];
    bounds_codes(p, valid, v);
    accumulate_bounds_codes(sa, v, valid, sim, uniform, bounds, s_red, kBoundsWords);
}

// Shared-memory scratch of finalize_grid (blockDim.x <= 256 for every caller).
constexpr uint32_t kFinalizeChunk = 64;   // simulations finalised per pass (at most)
struct FinalizeScratch {
    unsigned long long scan[256];
    uint32_t w[kFinalizeChunk][kBoundsWords];
    unsigned long long carry;
    unsigned long long boxes;   // boxes of all simulations (the max_boxes check)
    int bad;
};

// Run by the last CTA to finish: turn the bounds into each simulation's grid,
// choose its x sub-bins, assign its range of the box table, check capacity
// (boxes against max_boxes, table entries against table_capacity), and reset
// the accumulators for next time.
// `fs` may point into shared memory the CTA no longer needs.
__device__ __forceinline__ void finalize_grid(const SimArgs &sa, uint32_t *bounds,
                                              ug_grid_info *geo, Ctrl *ctrl, uint32_t max_boxes,
                                              int32_t *status, FinalizeScratch &fs) {
    unsigned long long *s_scan = fs.scan;
    constexpr uint32_t kChunk = kFinalizeChunk;
    uint32_t (*s_w)[kBoundsWords] = fs.w;
    unsigned long long &s_carry = fs.carry;
    int &s_bad = fs.bad;
    const int tid = threadIdx.x, nt = blockDim.x;
    const uint32_t copies = sa.bounds_copies;
    if (tid == 0) { s_carry = 0; s_bad = 0; fs.boxes = 0; }
    __syncthreads();
    const uint32_t chunk = min(kChunk, (uint32_t)nt);   // one thread per simulation
    for (uint32_t c0 = 0; c0 < sa.nsims; c0 += chunk) {
        const uint32_t nchunk = min(chunk, sa.nsims - c0);
        // max over the copies of every word of this chunk, all threads at once,
        // resetting the accumulators for the next use
        for (uint32_t q = tid; q < nchunk * kBoundsWords; q += nt) s_w[q / kBoundsWords][q % kBoundsWords] = 0u;
        __syncthreads();
        const uint32_t total_words = copies * nchunk * kBoundsWords;
        for (uint32_t q = tid; q < total_words; q += nt) {
            const uint32_t cp = q / (nchunk * kBoundsWords);
            const uint32_t rem = q - cp * nchunk * kBoundsWords;
            uint32_t *slot = &bounds[((size_t)cp * sa.nsims + c0) * kBoundsWords + rem];
            const uint32_t v = *(volatile uint32_t *)slot;
            *slot = 0u;
            if (v) atomicMax(&s_w[rem / kBoundsWords][rem % kBoundsWords], v);
        }
        __syncthreads();
        const uint32_t s = c0 + tid;
        unsigned long long nb = 0;
        ug_grid_info g{};
        if (tid < (int)nchunk) {
            const uint32_t a0 = sim_begin(sa, s), a1 = sim_end(sa, s);
            g.agent_base = a0;
            g.nagents = a1 - a0;
            if (a1 > a0) {
                uint32_t w[8];
                for (int k = 0; k < 8; ++k) w[k] = s_w[tid][k];
                const ug_params P = sim_params(sa, s);
                const float m2 = 2.0f * P.contact_margin;
                // edge = largest contact distance + 8 ulp of the largest
                // coordinate magnitude: float32 rounding of a box coordinate
                // moves an agent by at most ~3 such ulps, so no contact pair
                // (distance < largest contact distance) can end up two boxes apart
                const float S = __fadd_rn(ord_dec(w[6]), m2);
                float C = S;
                for (int a = 0; a < 3; ++a)
                    C = fmaxf(C, fmaxf(fabsf(ord_dec(w[a])), fabsf(ord_dec(w[3 + a]))));
                const float ulpC = __fsub_rn(__uint_as_float(__float_as_uint(C) + 1u), C);
                const float e = __fadd_rn(S, 8.0f * ulpC);
                const float mind = -ord_dec(w[7]);
                bool bad = !(e > 0.0f) || !isfinite(e) || !isfinite(C) || !(mind > 0.0f);
                g.edge = e;
                for (int a = 0; a < 3; ++a) {
                    const float lo = -ord_dec(w[a]);
                    const float hi = ord_dec(w[3 + a]);
                    const float o = __fsub_rn(lo, e);
                    const float f = floorf(__fdiv_rn(__fsub_rn(hi, o), e));
                    g.origin[a] = o;
                    if (!(f < 2097152.0f) || !isfinite(lo) || !isfinite(hi)) { bad = true; g.dims[a] = 3; }
                    else g.dims[a] = max((int)f, 1) + 2;
                }
                if (bad) { atomicOr(&s_bad, 1); nb = 0; }
                else nb = (unsigned long long)g.dims[0] * g.dims[1] * g.dims[2];
            }
        }
        // nb: boxes; the table holds K = 2^ks entries per box
        if (tid < (int)nchunk && nb) atomicAdd(&fs.boxes, nb);
        const int ks = tid < (int)nchunk ? sub_shift(g.nagents, nb) : 0;
        const unsigned long long nboxes = nb;
        nb <<= ks;
        // block exclusive scan of nb (Hillis-Steele on nt <= 256 entries)
        s_scan[tid] = nb;
        __syncthreads();
        for (int off = 1; off < nt; off <<= 1) {
            const unsigned long long add = tid >= off ? s_scan[tid - off] : 0ull;
            __syncthreads();
            s_scan[tid] += add;
            __syncthreads();
        }
        const unsigned long long incl = s_scan[tid];
        const unsigned long long base = s_carry + incl - nb;
        if (tid < (int)nchunk) {
            g.box_base = (uint32_t)min(base, 0xffffffffull);
            g.nboxes = (uint32_t)min(nboxes, 0xffffffffull);
            g.reserved = (uint32_t)ks;
            geo[s] = g;
        }
        __syncthreads();
        if (tid == nt - 1) s_carry += incl;
        __syncthreads();
    }
    if (tid == 0) {
        if (s_bad) set_status(status, UG_EBADSTATE);
        const unsigned long long total = s_carry;   // table entries
        const bool too_large = fs.boxes > (unsigned long long)max_boxes ||
                               total > table_capacity(sa.n, max_boxes);
        if (too_large) set_status(status, UG_EGRID_TOO_LARGE);
        ctrl->total_boxes = (s_bad || too_large) ? 0u : (uint32_t)total;
        ctrl->done = 0;
        __threadfence();
    }
}

// Last-CTA election after a grid-wide accumulation.  Every thread calls it.
__device__ __forceinline__ bool elect_last_cta(uint32_t *counter) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t prev = atomicAdd(counter, 1u);
        s_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// ------------------------------------------------------------------ workspace
struct Workspace {
    uint32_t *counts;      // [table_capacity]     zero between steps
    uint32_t *start;       // [table_capacity + 1] the box table (K entries per box)
    uint32_t *key;         // [n]
    uint32_t *rank;        // [n]
    uint32_t *tmp;         // [n]
    float4 *sorted;        // [n]
    uint32_t *perm2;       // [n]
    ug_grid_info *geo;     // [nsims]
    uint32_t *bounds;      // [copies * nsims * 8]
    uint32_t *tile_sum;    // [ntiles * kTileCopies * kTileSumStride]  zero between steps
    unsigned long long *acc;   // [2n][4] fixed-point force sums of the every-pair-once step: the
                               // other agents' contributions (zero between steps), then each
                               // agent's own sums
    Ctrl *ctrl;
    uint32_t ntiles;
    size_t bytes;
};

size_t layout_workspace(void *base, uint32_t n, uint32_t nsims, uint32_t max_boxes, Workspace *w);
// Symmetric pair evaluation (ug_symmetric.cu): forces of box-sorted rows with
// each pair evaluated once (forward) or from both sides, acc[4n] int64 scratch.
int run_symmetric(bool forward, const float4 *sorted, const uint32_t *start, const ug_grid_info *geo,
                  uint32_t n, const ug_params &p, unsigned long long *acc, float4 *force,
                  int32_t *status, cudaStream_t s);
// The paper's version ladder (ug_ladder.cu): forces of `state` (caller's order)
// into force[4n] float64, with head[max_boxes] and next[n] as scratch.
int run_ladder(int version, const float4 *state, uint32_t n, const SimArgs &sa, uint32_t max_boxes,
               const Workspace &w, uint32_t *head, uint32_t *next, double *force, int32_t *status,
               cudaStream_t s);
int device_sm_count();

// ------------------------------------------------------------------ launchers
// Grid build pieces (ug_grid.cu).  All asynchronous on `s`.
void launch_bounds(const float4 *st, const SimArgs &sa, const Workspace &w, ug_grid_info *geo,
                   uint32_t max_boxes, int32_t *status, cudaStream_t s);
void launch_key(const float4 *st, const SimArgs &sa, const Workspace &w, const ug_grid_info *geo,
                ug_grid_info *geo_save, int32_t *status, cudaStream_t s);
void launch_scan(const Workspace &w, uint32_t *start, uint32_t max_boxes, int32_t *status,
                 cudaStream_t s);
void launch_place(const Workspace &w, const uint32_t *start, uint32_t n, int32_t *status,
                  cudaStream_t s);
void launch_canon(const Workspace &w, const uint32_t *start, const float4 *st_in,
                  const uint32_t *perm_in, float4 *st_sorted, uint32_t *perm_out, uint32_t *sigma,
                  uint32_t n, int32_t *status, cudaStream_t s, uint32_t *skey = nullptr);
// The caller-facing per-box table and geometry of a single-simulation build.
void launch_box_table(const uint32_t *table, const ug_grid_info *geo, uint32_t *box_start,
                      ug_grid_info *info, uint32_t max_boxes, int32_t *status, cudaStream_t s);

// Sweep (ug_sweep.cu).
enum SweepMode { kSweepForce = 0, kSweepStep = 1, kSweepPairs = 2 };
struct SweepOut {
    float4 *force;          // kSweepForce: required; kSweepStep: optional save of F
    float4 *state_out;      // kSweepStep
    uint32_t *bounds;       // kSweepStep: next bounds accumulators
    ug_grid_info *geo_next; // kSweepStep: finalised geometry for the next step
    Ctrl *ctrl;
    uint32_t max_boxes;
    uint32_t *pair_count;   // kSweepPairs
    uint32_t *nbr;
    uint32_t max_per_agent;
};
void launch_sweep(int mode, const float4 *sorted, const uint32_t *start, const ug_grid_info *geo,
                  const SimArgs &sa, const SweepOut &out, int block, int32_t *status,
                  cudaStream_t s, const uint32_t *skey = nullptr);
// Fused step with symmetric pair evaluation (ug_symmetric.cu): pairs once into
// w.acc, then the move kernel (displacement, bounds, next grid) clears w.acc.
void launch_sym_step(const float4 *sorted, const uint32_t *start, const ug_grid_info *geo,
                     const SimArgs &sa, const SweepOut &out, unsigned long long *acc,
                     int32_t *status, cudaStream_t s, const uint32_t *skey, bool windowed);
// Two agents per lane (ug_sweep2.cu), force or step mode: one simulation with
// the neighbour-row windows (windowed) or the full runs, or many simulations
// (full runs).
void launch_sweep2(int mode, const float4 *sorted, const uint32_t *start, const ug_grid_info *geo,
                   const SimArgs &sa, const SweepOut &out, int32_t *status, cudaStream_t s,
                   const uint32_t *skey, bool windowed = false);
void launch_apply(const float4 *st_in, const float4 *force, uint32_t n, const ug_params &p,
                  float4 *st_out, float4 *disp_out, int32_t *status, cudaStream_t s);

// Full forward steps (ug_api.cu); used by ug_step, ug_step_batched and the adjoint.
struct StepSaves {          // per-step records for the adjoint (nullable)
    float4 *sorted;         // [nsteps][n]
    uint32_t *sigma;        // [nsteps][n] sorted slot -> input row
    uint32_t *start;        // [nsteps][start_stride], start_stride >= table_capacity + 1
    size_t start_stride;    // entries; a multiple of 64 so every table is 256-byte aligned
    float4 *force;          // [nsteps][n]
    ug_grid_info *geo;      // [nsteps][nsims]
};
int run_steps(float4 *state, uint32_t *perm, const SimArgs &sa, int nsteps, uint32_t max_boxes,
              const Workspace &w, int sweep_block, int agents_per_lane, const StepSaves *saves,
              int32_t *status, cudaStream_t s, cudaEvent_t const *events = nullptr,
              bool windowed = false);

}  // namespace ug
