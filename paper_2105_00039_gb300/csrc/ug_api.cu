// C ABI entry points (include/ugmech.h): argument checks, workspace layout and
// the per-step kernel sequence.  All device work is asynchronous on the
// caller's stream; nothing here allocates device memory.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <utility>

#include "ug_internal.cuh"

namespace ug {

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int device_sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 148;
    if (dev < 64 && cached[dev] > 0) return cached[dev];
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        sms = 148;
    if (dev < 64) cached[dev] = sms;
    return sms;
}

static uint32_t bounds_copies(uint32_t nsims) { return nsims == 1 ? kBoundsCopiesSingle : 1u; }

// Layout (base may be null to size only).  The first four regions (ctrl, tile
// sums, counts, bounds) are contiguous and are the only ones every call zeroes.
size_t layout_workspace(void *base, uint32_t n, uint32_t nsims, uint32_t max_boxes, Workspace *w) {
    size_t off = 0;
    char *b = static_cast<char *>(base);
    auto take = [&](size_t bytes) -> char * {
        char *p = b ? b + off : nullptr;
        off = align256(off + bytes);
        return p;
    };
    // the box table has up to table_capacity entries (boxes x their sub-bins)
    const size_t cap = (size_t)table_capacity(n, max_boxes);
    w->ctrl = reinterpret_cast<Ctrl *>(take(sizeof(Ctrl)));
    w->ntiles = std::max<uint32_t>(1u, (uint32_t)((cap + kScanTile - 1) / kScanTile));
    w->tile_sum = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * kTileSumStride * kTileCopies * (size_t)w->ntiles));
    w->counts = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * cap));
    w->bounds = reinterpret_cast<uint32_t *>(
        take(sizeof(uint32_t) * kBoundsWords * (size_t)bounds_copies(nsims) * nsims));
    const size_t zero_end = off;
    w->start = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (cap + 1)));
    w->key = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (size_t)n));
    w->rank = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (size_t)n));
    w->tmp = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (size_t)n));
    w->sorted = reinterpret_cast<float4 *>(take(sizeof(float4) * (size_t)n));
    w->perm2 = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (size_t)n));
    w->geo = reinterpret_cast<ug_grid_info *>(take(sizeof(ug_grid_info) * (size_t)nsims));
    // fixed-point sums of the every-pair-once step (zeroed by run_steps when used)
    w->acc = reinterpret_cast<unsigned long long *>(take(64 * (size_t)n));
    w->bytes = off;
    (void)zero_end;
    return off;
}

static size_t zero_bytes(const Workspace &w) {
    return (size_t)(reinterpret_cast<char *>(w.start) - reinterpret_cast<char *>(w.ctrl));
}

static int cuda_status(cudaError_t e) { return e == cudaSuccess ? UG_OK : UG_ECUDA; }
static int last_launch() { return cuda_status(cudaGetLastError()); }

int run_steps(float4 *state, uint32_t *perm, const SimArgs &sa, int nsteps, uint32_t max_boxes,
              const Workspace &w, int sweep_block, int agents_per_lane, const StepSaves *saves,
              int32_t *status, cudaStream_t s, cudaEvent_t const *events, bool windowed) {
    const uint32_t n = sa.n;
    auto mark = [&](int k) {
        if (events) cudaEventRecord(events[k], s);
    };
    if (cudaMemsetAsync(w.ctrl, 0, zero_bytes(w), s) != cudaSuccess) return UG_ECUDA;
    // the every-pair-once step adds the other agents' contributions into the
    // first half of w.acc; its move kernel leaves that half zero after each step
    if (agents_per_lane == 3 && cudaMemsetAsync(w.acc, 0, 32 * (size_t)n, s) != cudaSuccess)
        return UG_ECUDA;
    mark(0);
    launch_bounds(state, sa, w, w.geo, max_boxes, status, s);
    uint32_t *pcur = perm, *pnext = w.perm2;
    for (int t = 0; t < nsteps; ++t) {
        uint32_t *start = saves ? saves->start + (size_t)t * saves->start_stride : w.start;
        float4 *sorted = saves ? saves->sorted + (size_t)t * n : w.sorted;
        mark(1 + 5 * t);
        launch_key(state, sa, w, w.geo, saves ? saves->geo + (size_t)t * sa.nsims : nullptr,
                   status, s);
        mark(2 + 5 * t);
        launch_scan(w, start, max_boxes, status, s);
        mark(3 + 5 * t);
        launch_place(w, start, n, status, s);
        mark(4 + 5 * t);
        // the provisional ranks are consumed by the placement kernel, so their
        // buffer carries the sorted rows' sort keys from canon to the sweep
        launch_canon(w, start, state, pcur, sorted, pnext,
                     saves ? saves->sigma + (size_t)t * n : nullptr, n, status, s, w.rank);
        mark(5 + 5 * t);
        SweepOut o{};
        o.state_out = state;
        o.force = saves ? saves->force + (size_t)t * n : nullptr;
        o.bounds = w.bounds;
        o.geo_next = w.geo;
        o.ctrl = w.ctrl;
        o.max_boxes = max_boxes;
        if (agents_per_lane == 3)
            launch_sym_step(sorted, start, w.geo, sa, o, w.acc, status, s, w.rank, windowed);
        else if (agents_per_lane == 2)
            launch_sweep2(kSweepStep, sorted, start, w.geo, sa, o, status, s, w.rank, windowed);
        else
            launch_sweep(kSweepStep, sorted, start, w.geo, sa, o, sweep_block, status, s, w.rank);
        std::swap(pcur, pnext);
    }
    mark(1 + 5 * nsteps);
    if (pcur != perm && perm != nullptr)
        if (cudaMemcpyAsync(perm, pcur, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
            return UG_ECUDA;
    return last_launch();
}

// ------------------------------------------------------------------ helpers kernels
__global__ void k_iota(uint32_t *p, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}
__global__ void k_scatter_rows(const float4 *__restrict__ rows, const uint32_t *__restrict__ perm,
                               uint32_t n, float4 *__restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[__ldg(perm + i)] = __ldg(rows + i);
}
__global__ void k_gather_rows(const float4 *__restrict__ rows, const uint32_t *__restrict__ perm,
                              uint32_t n, float4 *__restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __ldg(rows + __ldg(perm + i));
}

}  // namespace ug

using namespace ug;

static inline bool aligned(const void *p, size_t a) {
    return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0;
}
static inline bool rows_ok(const void *p) { return p != nullptr && aligned(p, 16); }

extern "C" {

const char *ug_strerror(int status) {
    switch (status) {
    case UG_OK: return "ok";
    case UG_EINVAL: return "invalid argument";
    case UG_EBADSTATE: return "non-finite coordinate or diameter not finite and positive";
    case UG_EGRID_TOO_LARGE: return "grid needs more boxes than max_boxes";
    case UG_ECAPACITY: return "per-agent output list too short";
    case UG_EWORKSPACE: return "workspace too small";
    case UG_ETIMEOUT: return "reserved (device wait timed out)";
    case UG_ECUDA: return "CUDA runtime error";
    default: return "unknown status";
    }
}

int ug_version(void) { return 10000; }

size_t ug_workspace_bytes(uint32_t n, uint32_t nsims, uint32_t max_boxes) {
    Workspace w;
    return layout_workspace(nullptr, n, nsims == 0 ? 1 : nsims, max_boxes, &w);
}

int ug_grid_build(const float *state_in, const uint32_t *perm_in, uint32_t n, float contact_margin,
                  float *state_sorted, uint32_t *perm_sorted, uint32_t *box_start,
                  uint32_t max_boxes, ug_grid_info *info, void *ws, size_t ws_bytes,
                  int32_t *status, void *stream) {
    if (n == 0) return UG_OK;
    if (n > kMaxAgents) return UG_EINVAL;
    if (!rows_ok(state_in) || !rows_ok(state_sorted) || !perm_sorted || !box_start || !info ||
        !status || !ws || !aligned(ws, 256) || !aligned(box_start, 16) || max_boxes < 27 || max_boxes > 0x7fffff00u ||
        !(contact_margin >= 0.0f))
        return UG_EINVAL;
    Workspace w;
    if (layout_workspace(ws, n, 1, max_boxes, &w) > ws_bytes) return UG_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SimArgs sa{};
    sa.nsims = 1;
    sa.n = n;
    sa.pval.contact_margin = contact_margin;
    sa.bounds_copies = bounds_copies(1);
    if (cudaMemsetAsync(w.ctrl, 0, zero_bytes(w), s) != cudaSuccess) return UG_ECUDA;
    const float4 *in = reinterpret_cast<const float4 *>(state_in);
    launch_bounds(in, sa, w, w.geo, max_boxes, status, s);
    launch_key(in, sa, w, w.geo, nullptr, status, s);
    launch_scan(w, w.start, max_boxes, status, s);
    launch_place(w, w.start, n, status, s);
    launch_canon(w, w.start, in, perm_in, reinterpret_cast<float4 *>(state_sorted), perm_sorted,
                 nullptr, n, status, s);
    // the caller's per-box table (the first sub-bin entry of every box) and geometry
    launch_box_table(w.start, w.geo, box_start, info, max_boxes, status, s);
    return last_launch();
}

int ug_compute_forces(const float *state_sorted, const uint32_t *box_start, const ug_grid_info *info,
                      uint32_t n, ug_params p, float *force, int32_t *status, void *stream) {
    if (n == 0) return UG_OK;
    if (n > kMaxAgents) return UG_EINVAL;
    if (!rows_ok(state_sorted) || !box_start || !info || !rows_ok(force) || !status) return UG_EINVAL;
    SimArgs sa{};
    sa.nsims = 1;
    sa.n = n;
    sa.pval = p;
    sa.bounds_copies = 1;
    sa.per_box_table = true;   // the caller's table from ug_grid_build
    SweepOut o{};
    o.force = reinterpret_cast<float4 *>(force);
    launch_sweep2(kSweepForce, reinterpret_cast<const float4 *>(state_sorted), box_start, info, sa,
                  o, status, static_cast<cudaStream_t>(stream), nullptr);
    return last_launch();
}

int ug_list_pairs(const float *state_sorted, const uint32_t *box_start, const ug_grid_info *info,
                  uint32_t n, float contact_margin, uint32_t max_per_agent, uint32_t *count,
                  uint32_t *nbr, int32_t *status, void *stream) {
    if (n == 0) return UG_OK;
    if (n > kMaxAgents) return UG_EINVAL;
    if (!rows_ok(state_sorted) || !box_start || !info || !count || (!nbr && max_per_agent) ||
        !status)
        return UG_EINVAL;
    SimArgs sa{};
    sa.nsims = 1;
    sa.n = n;
    sa.pval.contact_margin = contact_margin;
    sa.bounds_copies = 1;
    sa.per_box_table = true;   // the caller's table from ug_grid_build
    SweepOut o{};
    o.pair_count = count;
    o.nbr = nbr;
    o.max_per_agent = max_per_agent;
    launch_sweep(kSweepPairs, reinterpret_cast<const float4 *>(state_sorted), box_start, info, sa, o,
                 128, status, static_cast<cudaStream_t>(stream));
    return last_launch();
}

int ug_apply_displacement(const float *state_in, const float *force, uint32_t n, ug_params p,
                          float *state_out, float *disp_out, int32_t *status, void *stream) {
    if (n == 0) return UG_OK;
    if (n > kMaxAgents) return UG_EINVAL;
    if (!rows_ok(state_in) || !rows_ok(force) || !rows_ok(state_out) ||
        (disp_out && !aligned(disp_out, 16)) || !status)
        return UG_EINVAL;
    launch_apply(reinterpret_cast<const float4 *>(state_in), reinterpret_cast<const float4 *>(force),
                 n, p, reinterpret_cast<float4 *>(state_out), reinterpret_cast<float4 *>(disp_out),
                 status, static_cast<cudaStream_t>(stream));
    return last_launch();
}

int ug_step(float *state, uint32_t *perm, uint32_t n, ug_params p, int32_t nsteps,
            uint32_t max_boxes, void *ws, size_t ws_bytes, int32_t *status, void *stream) {
    if (nsteps < 0) return UG_EINVAL;
    if (n == 0 || nsteps == 0) return UG_OK;
    if (n > kMaxAgents) return UG_EINVAL;
    if (!rows_ok(state) || !perm || !status || !ws || !aligned(ws, 256) || max_boxes < 27 || max_boxes > 0x7fffff00u ||
        !(p.contact_margin >= 0.0f))
        return UG_EINVAL;
    Workspace w;
    if (layout_workspace(ws, n, 1, max_boxes, &w) > ws_bytes) return UG_EWORKSPACE;
    SimArgs sa{};
    sa.nsims = 1;
    sa.n = n;
    sa.pval = p;
    sa.bounds_copies = bounds_copies(1);
    return run_steps(reinterpret_cast<float4 *>(state), perm, sa, nsteps, max_boxes, w, 128, 2,
                     nullptr, status, static_cast<cudaStream_t>(stream), nullptr,
                     windows_pay(n, max_boxes));
}

int ug_step_pairs_once(float *state, uint32_t *perm, uint32_t n, ug_params p, int32_t nsteps,
                       uint32_t max_boxes, void *ws, size_t ws_bytes, int32_t *status, void *stream) {
    if (nsteps < 0) return UG_EINVAL;
    if (n == 0 || nsteps == 0) return UG_OK;
    if (n > kMaxAgents) return UG_EINVAL;
    if (!rows_ok(state) || !perm || !status || !ws || !aligned(ws, 256) || max_boxes < 27 || max_boxes > 0x7fffff00u ||
        !(p.contact_margin >= 0.0f))
        return UG_EINVAL;
    Workspace w;
    if (layout_workspace(ws, n, 1, max_boxes, &w) > ws_bytes) return UG_EWORKSPACE;
    SimArgs sa{};
    sa.nsims = 1;
    sa.n = n;
    sa.pval = p;
    sa.bounds_copies = bounds_copies(1);
    return run_steps(reinterpret_cast<float4 *>(state), perm, sa, nsteps, max_boxes, w, 128, 3,
                     nullptr, status, static_cast<cudaStream_t>(stream), nullptr,
                     windows_pay_pairs_once(n, max_boxes));
}

int ug_step_traced(float *state, uint32_t *perm, uint32_t n, ug_params p, int32_t nsteps,
                   uint32_t max_boxes, void *ws, size_t ws_bytes, int32_t *status, void *stream,
                   void *const *events, int32_t nevents) {
    if (nsteps < 0 || !events || nevents < 2 + 5 * nsteps) return UG_EINVAL;
    if (n == 0 || nsteps == 0) return UG_OK;
    if (n > kMaxAgents) return UG_EINVAL;
    if (!rows_ok(state) || !perm || !status || !ws || !aligned(ws, 256) || max_boxes < 27 || max_boxes > 0x7fffff00u ||
        !(p.contact_margin >= 0.0f))
        return UG_EINVAL;
    Workspace w;
    if (layout_workspace(ws, n, 1, max_boxes, &w) > ws_bytes) return UG_EWORKSPACE;
    SimArgs sa{};
    sa.nsims = 1;
    sa.n = n;
    sa.pval = p;
    sa.bounds_copies = bounds_copies(1);
    return run_steps(reinterpret_cast<float4 *>(state), perm, sa, nsteps, max_boxes, w, 128, 2,
                     nullptr, status, static_cast<cudaStream_t>(stream),
                     reinterpret_cast<cudaEvent_t const *>(events), windows_pay(n, max_boxes));
}

int ug_step_batched(float *state, uint32_t *perm, const uint32_t *sim_offset, uint32_t nsims,
                    uint32_t n_total, const ug_params *params, int32_t nsteps, uint32_t max_boxes,
                    const ug_tuning *tuning, void *ws, size_t ws_bytes, int32_t *status,
                    void *stream) {
    if (nsteps < 0) return UG_EINVAL;
    if (n_total == 0 || nsteps == 0) return UG_OK;
    if (n_total > kMaxAgents) return UG_EINVAL;
    if (!rows_ok(state) || !perm || !sim_offset || nsims == 0 || !params || !status || !ws ||
        !aligned(ws, 256) || max_boxes < 27 || max_boxes > 0x7fffff00u)
        return UG_EINVAL;
    Workspace w;
    if (layout_workspace(ws, n_total, nsims, max_boxes, &w) > ws_bytes) return UG_EWORKSPACE;
    SimArgs sa{};
    sa.offset = sim_offset;
    sa.pdev = params;
    sa.nsims = nsims;
    sa.n = n_total;
    sa.bounds_copies = bounds_copies(nsims);
    const int block = tuning && tuning->sweep_block ? tuning->sweep_block : 128;
    const int apl = tuning && tuning->agents_per_lane ? tuning->agents_per_lane : 2;
    const int pair_mode = tuning ? tuning->pair_mode : 0;
    const int walk = tuning ? tuning->neighbour_walk : 0;
    if ((block != 64 && block != 128) || (apl != 1 && apl != 2) || (pair_mode != 0 && pair_mode != 1) ||
        walk < 0 || walk > 2)
        return UG_EINVAL;

    if (pair_mode == 1)   // every pair once: its own kernels, whatever the sweep layout
        return run_steps(reinterpret_cast<float4 *>(state), perm, sa, nsteps, max_boxes, w, 128, 3,
                         nullptr, status, static_cast<cudaStream_t>(stream), nullptr,
                         walk == 2 || (walk == 0 && windows_pay_pairs_once(n_total, max_boxes)));
    return run_steps(reinterpret_cast<float4 *>(state), perm, sa, nsteps, max_boxes, w, block, apl,
                     nullptr, status, static_cast<cudaStream_t>(stream), nullptr,
                     walk == 2 || (walk == 0 && windows_pay(n_total, max_boxes)));
}

int ug_tune_batched(const float *state, const uint32_t *sim_offset, uint32_t nsims, uint32_t n_total,
                    const ug_params *params, uint32_t max_boxes, ug_tuning *best, void *ws,
                    size_t ws_bytes, void *stream) {
    if (!best) return UG_EINVAL;
    memset(best, 0, sizeof(*best));
    best->sweep_block = 128;
    best->agents_per_lane = 2;
    if (n_total == 0) return UG_OK;
    if (n_total > kMaxAgents) return UG_EINVAL;
    if (!rows_ok(state) || !sim_offset || nsims == 0 || !params || !ws || !aligned(ws, 256) ||
        max_boxes < 27 || max_boxes > 0x7fffff00u)
        return UG_EINVAL;
    Workspace w;
    const size_t base = layout_workspace(ws, n_total, nsims, max_boxes, &w);
    const size_t rows_bytes = align256(sizeof(float4) * (size_t)n_total);
    const size_t ids_bytes = align256(sizeof(uint32_t) * (size_t)n_total);
    const size_t need = base + rows_bytes + ids_bytes + 256;
    if (need > ws_bytes) return UG_EWORKSPACE;
    // scratch copies of the rows and ids, advanced by a few fused steps per candidate
    char *extra = static_cast<char *>(ws) + base;
    float4 *rows = reinterpret_cast<float4 *>(extra);
    uint32_t *ids = reinterpret_cast<uint32_t *>(extra + rows_bytes);
    int32_t *status = reinterpret_cast<int32_t *>(extra + rows_bytes + ids_bytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SimArgs sa{};
    sa.offset = sim_offset;
    sa.pdev = params;
    sa.nsims = nsims;
    sa.n = n_total;
    sa.bounds_copies = bounds_copies(nsims);
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), s) != cudaSuccess) return UG_ECUDA;
    auto reset = [&]() -> int {
        if (cudaMemcpyAsync(rows, state, sizeof(float4) * (size_t)n_total, cudaMemcpyDeviceToDevice,
                            s) != cudaSuccess)
            return UG_ECUDA;
        k_iota<<<(n_total + 255) / 256, 256, 0, s>>>(ids, n_total);
        return last_launch();
    };
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return UG_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return UG_ECUDA; }
    // candidates: (agents per lane, threads per CTA, neighbour walk: 1 full runs,
    // 2 windows), and every pair once (3), each timed on kTuneSteps fused steps
    // (grid build + sweep + move) from the given rows, after one untimed step.
    // The windows serve the two-agent sweep of one simulation and every pair
    // once; the other layouts walk full runs.
    constexpr int kTuneSteps = 3;
    constexpr int kCands = 6;
    const int cands[kCands][3] = {{1, 64, 1}, {1, 128, 1}, {2, 128, 1}, {2, 128, 2}, {3, 128, 1},
                                  {3, 128, 2}};
    float best_ms = 1e30f;
    int rc = UG_OK;
    for (int c = 0; c < kCands && rc == UG_OK; ++c) {
        if (cands[c][0] == 2 && cands[c][2] == 2 && nsims > 1) continue;
        const bool win = cands[c][2] == 2;
        rc = reset();
        if (rc == UG_OK)
            rc = run_steps(rows, ids, sa, 1, max_boxes, w, cands[c][1], cands[c][0], nullptr, status, s,
                           nullptr, win);
        if (rc == UG_OK) rc = reset();
        if (rc != UG_OK) break;
        cudaEventRecord(e0, s);
        rc = run_steps(rows, ids, sa, kTuneSteps, max_boxes, w, cands[c][1], cands[c][0], nullptr,
                       status, s, nullptr, win);
        cudaEventRecord(e1, s);
        if (rc != UG_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = UG_ECUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best->pair_mode = cands[c][0] == 3 ? 1 : 0;
            best->agents_per_lane = cands[c][0] == 3 ? 2 : cands[c][0];
            best->sweep_block = cands[c][1];
            best->neighbour_walk = cands[c][0] == 1 ? 0 : cands[c][2];
        }
    }
    int32_t hst = 0;
    if (rc == UG_OK && cudaMemcpy(&hst, status, sizeof(hst), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = UG_ECUDA;
    if (rc == UG_OK && hst != 0) rc = hst;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == UG_OK) rc = last_launch();
    return rc;
}

size_t ug_ladder_workspace_bytes(uint32_t n, uint32_t max_boxes) {
    Workspace w;
    return layout_workspace(nullptr, n, 1, max_boxes, &w) + align256(sizeof(uint32_t) * (size_t)max_boxes) +
           align256(sizeof(uint32_t) * (size_t)n);
}

int ug_forces_ladder(int32_t version, const float *state, uint32_t n, ug_params p,
                     uint32_t max_boxes, double *force, void *ws, size_t ws_bytes, int32_t *status,
                     void *stream) {
    if (version < 0 || version > 3) return UG_EINVAL;
    if (n == 0) return UG_OK;
    if (n > kMaxAgents) return UG_EINVAL;
    if (!rows_ok(state) || !force || !aligned(force, 16) || !status || !ws || !aligned(ws, 256) ||
        max_boxes < 27 || max_boxes > 0x7fffff00u || !(p.contact_margin >= 0.0f))
        return UG_EINVAL;
    if (ug_ladder_workspace_bytes(n, max_boxes) > ws_bytes) return UG_EWORKSPACE;
    Workspace w;
    const size_t base = layout_workspace(ws, n, 1, max_boxes, &w);
    uint32_t *head = reinterpret_cast<uint32_t *>(static_cast<char *>(ws) + base);
    uint32_t *next = reinterpret_cast<uint32_t *>(static_cast<char *>(ws) + base +
                                                  align256(sizeof(uint32_t) * (size_t)max_boxes));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(w.ctrl, 0, zero_bytes(w), s) != cudaSuccess) return UG_ECUDA;
    SimArgs sa{};
    sa.nsims = 1;
    sa.n = n;
    sa.pval = p;
    sa.bounds_copies = bounds_copies(1);
    return run_ladder(version, reinterpret_cast<const float4 *>(state), n, sa, max_boxes, w, head,
                      next, force, status, s);
}

int ug_forces_symmetric(int32_t each_pair_once, const float *state_sorted, const uint32_t *box_start,
                        const ug_grid_info *info, uint32_t n, ug_params p, float *force, void *ws,
                        size_t ws_bytes, int32_t *status, void *stream) {
    if (n == 0) return UG_OK;
    if (n > kMaxAgents) return UG_EINVAL;
    if (!rows_ok(state_sorted) || !box_start || !info || !rows_ok(force) || !status || !ws ||
        !aligned(ws, 256))
        return UG_EINVAL;
    if (ws_bytes < 32 * (size_t)n) return UG_EWORKSPACE;
    return run_symmetric(each_pair_once != 0, reinterpret_cast<const float4 *>(state_sorted), box_start,
                         info, n, p, static_cast<unsigned long long *>(ws),
                         reinterpret_cast<float4 *>(force), status, static_cast<cudaStream_t>(stream));
}

int ug_iota(uint32_t *perm, uint32_t n, void *stream) {
    if (n == 0) return UG_OK;
    if (n > kMaxAgents) return UG_EINVAL;
    if (!perm) return UG_EINVAL;
    k_iota<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(perm, n);
    return last_launch();
}

int ug_scatter_rows(const float *rows, const uint32_t *perm, uint32_t n, float *rows_by_id,
                    void *stream) {
    if (n == 0) return UG_OK;
    if (n > kMaxAgents) return UG_EINVAL;
    if (!rows_ok(rows) || !perm || !rows_ok(rows_by_id)) return UG_EINVAL;
    k_scatter_rows<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float4 *>(rows), perm, n, reinterpret_cast<float4 *>(rows_by_id));
    return last_launch();
}

int ug_gather_rows(const float *rows_by_id, const uint32_t *perm, uint32_t n, float *rows,
                   void *stream) {
    if (n == 0) return UG_OK;
    if (n > kMaxAgents) return UG_EINVAL;
    if (!rows_ok(rows_by_id) || !perm || !rows_ok(rows)) return UG_EINVAL;
    k_gather_rows<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float4 *>(rows_by_id), perm, n, reinterpret_cast<float4 *>(rows));
    return last_launch();
}

}  // extern "C"
