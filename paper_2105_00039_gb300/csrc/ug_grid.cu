// Uniform-grid construction (Hesam et al., Sec. IV-A and IV-D), GB300 design.
//
// The paper keeps a per-box count plus a linked list of agents and sorts agent
// state along a Z-order curve so that neighbours share cache lines.  Here the
// grid IS the sort: a counting sort by box key, boxes in row-major order (x
// fastest, so the three boxes of a neighbourhood along x are one contiguous
// run), agents of a box by x sub-bin (K = 2^ks slices of the box edge along x,
// ks chosen per simulation from its density; see sort_key) and, within a
// sub-bin, in their input order.  The table therefore has K entries per box,
// one per sub-bin.  Five kernels per rebuild:
//
//   k_bounds  (first step only; later steps get it from the sweep epilogue)
//             per-simulation min/max corner and max diameter -> grid geometry
//   k_key     sort key (box and x sub-bin) of every row + warp-aggregated
//             atomic histogram; the atomic's return value is a provisional
//             rank inside the sub-bin; the rows of every scan tile (8192 table
//             entries) are summed on the side
//   k_scan    exclusive scan of the sub-bin counts, one CTA per tile, whose
//             prefix is the sum of the earlier tiles' row counts (no inter-CTA
//             wait), also re-zeroing the counts
//   k_place   row index -> provisional slot; re-zeroes the tile sums
//   k_canon   stable order inside each sub-bin (rank = rows of the sub-bin
//             with a smaller input index), gathering rows and ids into that slot
#include <cuda_runtime.h>

#include <algorithm>

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
    __shared__ FinalizeScratch fs;
    if (elect_last_cta(&ctrl->done)) finalize_grid(sa, bounds, geo, ctrl, max_boxes, status, fs);
}

// ------------------------------------------------------------------ key + histogram
// Each warp covers 2 x 32 consecutive rows (kKeyItems chunks), so that two
// independent chains of loads and atomics are in flight per thread.
constexpr int kKeyItems = 2;
constexpr int kKeyWarps = 8;   // 256 threads
constexpr int kTilePairs = 3;  // tile sums added by lane 0 per warp and row chunk

__global__ void __launch_bounds__(kKeyWarps * 32)
k_key(const float4 *__restrict__ st, SimArgs sa, const ug_grid_info *__restrict__ geo,
      uint32_t *counts, uint32_t *tile_sum, uint32_t *__restrict__ key,
      uint32_t *__restrict__ rank, ug_grid_info *geo_save, int32_t *status) {
    chain_begin();
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t stride = gridDim.x * blockDim.x;
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
    uint32_t k[kKeyItems], base[kKeyItems];
    int myhead[kKeyItems], nrun[kKeyItems];
#pragma unroll
    for (int it = 0; it < kKeyItems; ++it) {
        k[it] = 0xffffffffu;
        if (idx[it] < sa.n) {
            const uint32_t sim = uniform ? csim : find_sim(sa, idx[it]);
            k[it] = sort_key(p[it], geo[sim]);
        }
        // rows arrive nearly sorted by box (the previous step's order), so equal
        // keys mostly sit on consecutive lanes: each run of equal keys takes one
        // atomic, and its lanes get consecutive provisional ranks
        const uint32_t prevk = __shfl_up_sync(kFull, k[it], 1);
        const bool head = lane == 0 || prevk != k[it];
        const unsigned heads = __ballot_sync(kFull, head);
        myhead[it] = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
        const unsigned after = lane == 31 ? 0u : heads & (0xffffffffu << (lane + 1));
        nrun[it] = head && idx[it] < sa.n ? (after ? __ffs(after) - 1 : 32) - lane : 0;
    }
    // all the histogram atomics first, so that their round trips overlap
#pragma unroll
    for (int it = 0; it < kKeyItems; ++it)
        base[it] = nrun[it] > 0 ? atomicAdd(&counts[k[it]], (uint32_t)nrun[it]) : 0u;
    // rows per scan tile, added into this warp's copy of the tile sums: lane 0
    // adds the rows of up to kTilePairs tiles (rows move between boxes every
    // step, so a warp often holds rows of the tiles either side of its own);
    // lanes of any further tile (rare) add their own rows
    const uint32_t copy = (blockIdx.x * kKeyWarps + (threadIdx.x >> 5)) % kTileCopies;
    auto tile_add = [&](uint32_t t, uint32_t rows) {
        atomicAdd(&tile_sum[(t * kTileCopies + copy) * kTileSumStride], rows);
    };
#pragma unroll
    for (int it = 0; it < kKeyItems; ++it) {
        const bool valid = idx[it] < sa.n;
        const uint32_t tl = k[it] >> kScanTileShift;
        unsigned rest = __ballot_sync(kFull, valid);
#pragma unroll
        for (int j = 0; j < kTilePairs; ++j) {
            if (rest) {
                const uint32_t tj = __shfl_sync(kFull, tl, __ffs(rest) - 1);
                const unsigned mj = __ballot_sync(kFull, valid && tl == tj);
                rest &= ~mj;
                if (lane == 0) tile_add(tj, (uint32_t)__popc(mj));
            }
        }
        if ((rest >> lane) & 1u) tile_add(tl, 1u);
    }
#pragma unroll
    for (int it = 0; it < kKeyItems; ++it) {
        const uint32_t b = __shfl_sync(kFull, base[it], myhead[it]);
        if (idx[it] < sa.n) {
            rank[idx[it]] = b + (uint32_t)(lane - myhead[it]);
            key[idx[it]] = k[it];
        }
    }
}

// ------------------------------------------------------------------ tile scan
// CTA t scans boxes [t * kScanTile, (t + 1) * kScanTile).  Its exclusive
// prefix, the rows in all earlier boxes, is the sum of the earlier tiles' row
// counts that k_key accumulated (all copies), so no CTA waits on another.
__global__ void __launch_bounds__(kScanThreads)
k_scan(uint32_t *__restrict__ counts, uint32_t *__restrict__ start, const Ctrl *ctrl,
       const uint32_t *__restrict__ tile_sum, int32_t *status) {
    __shared__ uint32_t s_warp[kScanThreads / 32];
    __shared__ uint32_t s_pre[kScanThreads / 32];
    chain_begin();
    if (cta_failed(status)) return;
    const uint32_t B = *(volatile const uint32_t *)&ctrl->total_boxes;
    const uint32_t ntiles = (B + kScanTile - 1) / kScanTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t t = blockIdx.x;
    if (t >= ntiles) return;
    {
        uint32_t pre = 0;
        for (uint32_t u = threadIdx.x; u < t * kTileCopies; u += kScanThreads)
            pre += __ldg(tile_sum + (size_t)u * kTileSumStride);
        pre = __reduce_add_sync(kFull, pre);
        if (lane == 0) s_pre[warp] = pre;
    }
    {
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
        uint32_t excl = 0;
#pragma unroll
        for (int w = 0; w < kScanThreads / 32; ++w) excl += s_pre[w];
        uint32_t run = excl + wbase + inc - tsum;
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
        if (t == ntiles - 1 && threadIdx.x == 0) start[B] = excl + tile_total;
    }
}

// ------------------------------------------------------------------ placement
__global__ void __launch_bounds__(256)
k_place(const uint32_t *__restrict__ key, const uint32_t *__restrict__ rank,
        const uint32_t *__restrict__ start, uint32_t *__restrict__ tmp, uint32_t n,
        uint32_t *__restrict__ tile_sum, uint32_t ntiles, int32_t *status) {
    chain_begin();
    // the scan has consumed the tile sums: clear them for the next rebuild
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles * kTileCopies;
         t += gridDim.x * blockDim.x)
        tile_sum[(size_t)t * kTileSumStride] = 0u;
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
        // stable rank inside the sub-bin: its rows with a smaller input index
        uint32_t r = 0;
        for (uint32_t t = b0[q]; t < b1[q]; ++t) r += __ldg(tmp + t) < id[q];
        const uint32_t dest = b0[q] + r;
        st_out[dest] = row[q];
        perm_out[dest] = pid[q];
        if (sigma) sigma[dest] = id[q];
        if (skey) skey[dest] = k[q];
    }
}

// ------------------------------------------------------------------ per-box table
// The table of a single simulation reduced to one entry per box (entry b << ks,
// the start of the box's first sub-bin; the last entry is n), and its geometry
// with reserved = 0, which is how callers of the per-box entry points read a
// box table.  Writes the geometry even after a failed build.
__global__ void __launch_bounds__(256)
k_box_table(const uint32_t *__restrict__ table, const ug_grid_info *__restrict__ geo,
            uint32_t *__restrict__ box_start, ug_grid_info *info, int32_t *status) {
    chain_begin();
    const ug_grid_info g = geo[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ug_grid_info o = g;
        o.reserved = 0u;
        info[0] = o;
    }
    if (cta_failed(status)) return;
    const int ks = grid_shift(g);
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= g.nboxes; b += gridDim.x * blockDim.x)
        box_start[b] = __ldg(table + ((size_t)b << ks));
}

// ------------------------------------------------------------------ launchers
static inline unsigned blocks_for(uint32_t n, int t) { return (unsigned)((n + t - 1) / t); }

void launch_bounds(const float4 *st, const SimArgs &sa, const Workspace &w, ug_grid_info *geo,
                   uint32_t max_boxes, int32_t *status, cudaStream_t s) {
    launch_chained(k_bounds, blocks_for(sa.n, 256), 256, s, st, sa, w.bounds, geo, w.ctrl,
                   max_boxes, status);
}

void launch_key(const float4 *st, const SimArgs &sa, const Workspace &w, const ug_grid_info *geo,
                ug_grid_info *geo_save, int32_t *status, cudaStream_t s) {
    launch_chained(k_key, blocks_for(sa.n, kKeyWarps * 32 * kKeyItems), kKeyWarps * 32, s, st, sa, geo, w.counts, w.tile_sum,
                   w.key, w.rank, geo_save, status);
}

void launch_scan(const Workspace &w, uint32_t *start, uint32_t max_boxes, int32_t *status,
                 cudaStream_t s) {
    (void)max_boxes;
    launch_chained(k_scan, w.ntiles, (unsigned)kScanThreads, s, w.counts, start,
                   (const Ctrl *)w.ctrl, (const uint32_t *)w.tile_sum, status);
}

void launch_place(const Workspace &w, const uint32_t *start, uint32_t n, int32_t *status,
                  cudaStream_t s) {
    launch_chained(k_place, blocks_for(n, 512), 256, s, w.key, w.rank, start, w.tmp, n, w.tile_sum,
                   w.ntiles, status);
}

void launch_canon(const Workspace &w, const uint32_t *start, const float4 *st_in,
                  const uint32_t *perm_in, float4 *st_sorted, uint32_t *perm_out, uint32_t *sigma,
                  uint32_t n, int32_t *status, cudaStream_t s, uint32_t *skey) {
    launch_chained(k_canon, blocks_for(n, 512), 256, s, w.tmp, w.key, start, st_in, perm_in,
                   st_sorted, perm_out, sigma, n, skey, status);
}

}  // namespace ug

namespace ug {
void launch_box_table(const uint32_t *table, const ug_grid_info *geo, uint32_t *box_start,
                      ug_grid_info *info, uint32_t max_boxes, int32_t *status, cudaStream_t s) {
    const unsigned cap = 4u * (unsigned)device_sm_count();
    const unsigned blocks = (unsigned)std::min<size_t>(cap, ((size_t)max_boxes + 256) / 256);
    launch_chained(k_box_table, blocks, 256u, s, table, geo, box_start, info, status);
}
}  // namespace ug
