// Uniform-grid construction (Hesam et al., Sec. IV-A and IV-D), GB300 design.
//
// The paper keeps a per-box count plus a linked list of agents and sorts agent
// state along a Z-order curve so that neighbours share cache lines.  Here the
// grid IS the sort: a counting sort by box key, boxes in row-major order (x
// fastest, so the three boxes of a neighbourhood along x are one contiguous
// run), agents of a box in their input order.  Five kernels per rebuild:
//
//   k_bounds  (first step only; later steps get it from the sweep epilogue)
//             per-simulation min/max corner and max diameter -> grid geometry
//   k_key     box key of every row + warp-aggregated atomic histogram; the
//             atomic's return value is a provisional rank inside the box
//   k_scan    single-pass exclusive scan of the box counts with a warp-wide
//             decoupled look-back (bounded spins), also re-zeroing the counts
//   k_place   row index -> provisional slot
//   k_canon   stable order inside each box (rank = rows of the box with a
//             smaller input index), gathering rows and ids into that slot
#include <cuda_runtime.h>

#include <atomic>

#include "ug_internal.cuh"

namespace ug {

// ------------------------------------------------------------------ bounds
__global__ void __launch_bounds__(256)
k_bounds(const float4 *__restrict__ st, SimArgs sa, uint32_t *bounds, ug_grid_info *geo,
         Ctrl *ctrl, uint32_t max_boxes, int32_t *status) {
    chain_begin();
    if (cta_failed(status)) return;
    const uint32_t first = blockIdx.x * blockDim.x;
    const uint32_t i = first + threadIdx.x;
    const bool valid = i < sa.n;
    bool uniform;
    const uint32_t sim = cta_sim(sa, first, i, uniform);
    const float4 p = valid ? __ldg(st + i) : make_float4(0.f, 0.f, 0.f, 1.f);
    accumulate_bounds(sa, p, valid, sim, uniform, bounds, status);
    if (elect_last_cta(&ctrl->done)) finalize_grid(sa, bounds, geo, ctrl, max_boxes, status);
}

// ------------------------------------------------------------------ key + histogram
// Each warp covers 2 x 32 consecutive rows (kKeyItems chunks), so that two
// independent chains of loads and atomics are in flight per thread.
constexpr int kKeyItems = 2;

__global__ void __launch_bounds__(256)
k_key(const float4 *__restrict__ st, SimArgs sa, const ug_grid_info *__restrict__ geo,
      Ctrl *ctrl, uint32_t *counts, uint32_t *__restrict__ key, uint32_t *__restrict__ rank,
      unsigned long long *scan_status, uint32_t ntiles, ug_grid_info *geo_save,
      int32_t *status) {
    chain_begin();
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t t = gtid; t < ntiles; t += stride) scan_status[t] = 0ull;
    if (gtid == 0) ctrl->scan_ticket = 0u;
    if (geo_save)
        for (uint32_t s = gtid; s < sa.nsims; s += stride) geo_save[s] = geo[s];
    if (cta_failed(status)) return;

    const int lane = threadIdx.x & 31;
    const uint32_t first = blockIdx.x * blockDim.x * kKeyItems;
    const uint32_t wbase = first + (threadIdx.x >> 5) * 32u * kKeyItems;
    bool uniform;
    const uint32_t csim = cta_sim_range(sa, first, blockDim.x * kKeyItems, uniform);
    float4 p[kKeyItems];
    uint32_t idx[kKeyItems];
#pragma unroll
    for (int it = 0; it < kKeyItems; ++it) {
        idx[it] = wbase + 32u * it + lane;
        p[it] = idx[it] < sa.n ? __ldg(st + idx[it]) : make_float4(0.f, 0.f, 0.f, 1.f);
    }
#pragma unroll
    for (int it = 0; it < kKeyItems; ++it) {
        const uint32_t i = idx[it];
        const bool valid = i < sa.n;
        uint32_t k = 0xffffffffu;
        if (valid) {
            const uint32_t sim = uniform ? csim : find_sim(sa, i);
            const ug_grid_info g = geo[sim];
            int bx, by, bz;
            k = box_key(p[it], g, bx, by, bz);
        }
        // rows arrive nearly sorted by box (the previous step's order), so equal
        // keys mostly sit on consecutive lanes: each run of equal keys takes one
        // atomic, and its lanes get consecutive provisional ranks
        const uint32_t prevk = __shfl_up_sync(kFull, k, 1);
        const bool head = lane == 0 || prevk != k;
        const unsigned heads = __ballot_sync(kFull, head);
        const int myhead = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
        const unsigned after = lane == 31 ? 0u : heads & (0xffffffffu << (lane + 1));
        const int nexthead = after ? __ffs(after) - 1 : 32;
        uint32_t base = 0;
        if (head && valid) base = atomicAdd(&counts[k], (uint32_t)(nexthead - lane));
        base = __shfl_sync(kFull, base, myhead);
        if (valid) {
            rank[i] = base + (uint32_t)(lane - myhead);
            key[i] = k;
        }
    }
}

// ------------------------------------------------------------------ look-back scan
// Tile status word: flag << 32 | value; flag 0 = not ready, 1 = tile sum only,
// 2 = inclusive prefix of everything up to and including the tile.
__device__ __forceinline__ void publish(unsigned long long *st, uint32_t t, uint32_t flag,
                                        uint32_t val) {
    *(volatile unsigned long long *)(st + t) = ((unsigned long long)flag << 32) | val;
}

// Exclusive prefix of tile t from its predecessors' status words, read by one
// warp 32 tiles at a time (lane l looks at tile t-1-l): sum tile aggregates
// back to the nearest tile that already knows its inclusive prefix.  Waits are
// bounded; on timeout the error is recorded and the partial sum returned so
// that successors finish too.
__device__ uint32_t look_back_warp(unsigned long long *st, uint32_t t, uint32_t spin_limit,
                                   int32_t *status) {
    const int lane = threadIdx.x & 31;
    uint32_t excl = 0;
    int j = (int)t - 1 - lane;
    uint32_t spins = 0;
    for (;;) {
        const unsigned long long w =
            j >= 0 ? *(volatile unsigned long long *)(st + j) : (2ull << 32);
        const uint32_t flag = (uint32_t)(w >> 32);
        if (__any_sync(kFull, flag == 0u)) {
            if (++spins > spin_limit || peek_status(status) != 0) {
                set_status(status, UG_ETIMEOUT);
                return excl;
            }
            __nanosleep(32);
            continue;
        }
        const unsigned pmask = __ballot_sync(kFull, flag == 2u);
        const int first = pmask ? __ffs(pmask) - 1 : 31;
        excl += __reduce_add_sync(kFull, lane <= first ? (uint32_t)w : 0u);
        if (pmask) return excl;
        j -= 32;
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan(uint32_t *__restrict__ counts, uint32_t *__restrict__ start, Ctrl *ctrl,
       unsigned long long *tstat, uint32_t spin_limit, int32_t *status) {
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ uint32_t s_warp[kScanThreads / 32];
    chain_begin();
    if (cta_failed(status)) return;
    const uint32_t B = *(volatile uint32_t *)&ctrl->total_boxes;
    const uint32_t ntiles = (B + kScanTile - 1) / kScanTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&ctrl->scan_ticket, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= ntiles) break;
        const uint32_t base = t * kScanTile + threadIdx.x * kScanItems;
        uint32_t v[kScanItems];
        if (base + kScanItems <= B) {
#pragma unroll
            for (int q = 0; q < kScanItems / 4; ++q) {
                const uint4 a = *reinterpret_cast<const uint4 *>(counts + base + 4 * q);
                v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kScanItems; ++k) v[k] = base + k < B ? counts[base + k] : 0u;
        }
        uint32_t tsum = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) tsum += v[k];
        // warp inclusive scan of thread sums
        uint32_t inc = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        uint32_t wbase = 0, tile_total = 0;
#pragma unroll
        for (int w = 0; w < kScanThreads / 32; ++w) {
            const uint32_t x = s_warp[w];
            if (w < warp) wbase += x;
            tile_total += x;
        }
        if (warp == 0) {
            uint32_t excl = 0;
            if (t == 0) {
                if (lane == 0) publish(tstat, t, 2u, tile_total);
            } else {
                if (lane == 0) publish(tstat, t, 1u, tile_total);
                excl = look_back_warp(tstat, t, spin_limit, status);
                if (lane == 0) publish(tstat, t, 2u, excl + tile_total);
            }
            if (lane == 0) s_prefix = excl;
        }
        __syncthreads();
        uint32_t run = s_prefix + wbase + inc - tsum;
        if (base + kScanItems <= B) {
#pragma unroll
            for (int q = 0; q < kScanItems / 4; ++q) {
                uint4 a;
                a.x = run; run += v[4 * q];
                a.y = run; run += v[4 * q + 1];
                a.z = run; run += v[4 * q + 2];
                a.w = run; run += v[4 * q + 3];
                *reinterpret_cast<uint4 *>(start + base + 4 * q) = a;
                *reinterpret_cast<uint4 *>(counts + base + 4 * q) = make_uint4(0u, 0u, 0u, 0u);
            }
        } else {
#pragma unroll
            for (int k = 0; k < kScanItems; ++k) {
                if (base + k < B) {
                    start[base + k] = run;
                    counts[base + k] = 0u;
                }
                run += v[k];
            }
        }
        if (t == ntiles - 1 && threadIdx.x == 0) start[B] = s_prefix + tile_total;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ placement
__global__ void __launch_bounds__(256)
k_place(const uint32_t *__restrict__ key, const uint32_t *__restrict__ rank,
        const uint32_t *__restrict__ start, uint32_t *__restrict__ tmp, uint32_t n,
        int32_t *status) {
    chain_begin();
    if (cta_failed(status)) return;
    const uint32_t i0 = blockIdx.x * blockDim.x * 2u + threadIdx.x, i1 = i0 + blockDim.x;
    uint32_t k0 = 0, k1 = 0, r0 = 0, r1 = 0;
    if (i0 < n) { k0 = __ldg(key + i0); r0 = __ldg(rank + i0); }
    if (i1 < n) { k1 = __ldg(key + i1); r1 = __ldg(rank + i1); }
    if (i0 < n) tmp[__ldg(start + k0) + r0] = i0;
    if (i1 < n) tmp[__ldg(start + k1) + r1] = i1;
}

__global__ void __launch_bounds__(256)
k_canon(const uint32_t *__restrict__ tmp, const uint32_t *__restrict__ key,
        const uint32_t *__restrict__ start, const float4 *__restrict__ st_in,
        const uint32_t *__restrict__ perm_in, float4 *__restrict__ st_out,
        uint32_t *__restrict__ perm_out, uint32_t *__restrict__ sigma, uint32_t n,
        uint32_t *__restrict__ skey, int32_t *status) {
    chain_begin();
    if (cta_failed(status)) return;
    // two slots per thread, their load chains interleaved
    uint32_t sl[2], id[2], k[2], b0[2], b1[2];
    sl[0] = blockIdx.x * blockDim.x * 2u + threadIdx.x;
    sl[1] = sl[0] + blockDim.x;
#pragma unroll
    for (int q = 0; q < 2; ++q) id[q] = sl[q] < n ? __ldg(tmp + sl[q]) : 0u;
#pragma unroll
    for (int q = 0; q < 2; ++q) k[q] = sl[q] < n ? __ldg(key + id[q]) : 0u;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        b0[q] = sl[q] < n ? __ldg(start + k[q]) : 0u;
        b1[q] = sl[q] < n ? __ldg(start + k[q] + 1) : 0u;
    }
    float4 row[2];
    uint32_t pid[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (sl[q] < n) {
            row[q] = __ldg(st_in + id[q]);
            pid[q] = perm_in ? __ldg(perm_in + id[q]) : id[q];
        }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (sl[q] >= n) continue;
        // stable rank inside the box: rows of the box with a smaller input index
        uint32_t r = 0;
        for (uint32_t t = b0[q]; t < b1[q]; ++t) r += __ldg(tmp + t) < id[q];
        const uint32_t dest = b0[q] + r;
        st_out[dest] = row[q];
        perm_out[dest] = pid[q];
        if (sigma) sigma[dest] = id[q];
        if (skey) skey[dest] = k[q];
    }
}

// ------------------------------------------------------------------ launchers
static inline unsigned blocks_for(uint32_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Bound on the look-back polls of the scan, process-wide (see ug_debug_spin_limit).
static std::atomic<uint32_t> g_spin_limit{kSpinLimit};
uint32_t spin_limit() { return g_spin_limit.load(std::memory_order_relaxed); }
uint32_t set_spin_limit(uint32_t v) { return g_spin_limit.exchange(v); }

void launch_bounds(const float4 *st, const SimArgs &sa, const Workspace &w, ug_grid_info *geo,
                   uint32_t max_boxes, int32_t *status, cudaStream_t s) {
    launch_chained(k_bounds, blocks_for(sa.n, 256), 256, s, st, sa, w.bounds, geo, w.ctrl,
                   max_boxes, status);
}

void launch_key(const float4 *st, const SimArgs &sa, const Workspace &w, const ug_grid_info *geo,
                ug_grid_info *geo_save, int32_t *status, cudaStream_t s) {
    launch_chained(k_key, blocks_for(sa.n, 256 * kKeyItems), 256, s, st, sa, geo, w.ctrl, w.counts, w.key,
                   w.rank, w.scan_status, w.ntiles, geo_save, status);
}

void launch_scan(const Workspace &w, uint32_t *start, uint32_t max_boxes, int32_t *status,
                 cudaStream_t s) {
    (void)max_boxes;
    const unsigned grid = (unsigned)min((int)w.ntiles, 2 * device_sm_count());
    launch_chained(k_scan, grid > 0 ? grid : 1u, (unsigned)kScanThreads, s, w.counts, start, w.ctrl,
                   w.scan_status, spin_limit(), status);
}

void launch_place(const Workspace &w, const uint32_t *start, uint32_t n, int32_t *status,
                  cudaStream_t s) {
    launch_chained(k_place, blocks_for(n, 512), 256, s, w.key, w.rank, start, w.tmp, n, status);
}

void launch_canon(const Workspace &w, const uint32_t *start, const float4 *st_in,
                  const uint32_t *perm_in, float4 *st_sorted, uint32_t *perm_out, uint32_t *sigma,
                  uint32_t n, int32_t *status, cudaStream_t s, uint32_t *skey) {
    launch_chained(k_canon, blocks_for(n, 512), 256, s, w.tmp, w.key, start, st_in, perm_in,
                   st_sorted, perm_out, sigma, n, skey, status);
}

}  // namespace ug
