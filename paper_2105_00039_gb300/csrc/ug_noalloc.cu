// Grid build that allocates nothing: its scratch space is a fixed array of
// device memory compiled into the library, for callers that cannot allocate.
//
// Who needs it: a caller that is handed only its inputs and outputs and may not
// allocate device memory at the point of the call -- for instance a plug-in
// whose host application owns every byte of the GPU's memory, or code that runs
// under a fixed memory budget.  Such a caller cannot supply the workspace that
// ug_grid_build asks for, so this variant brings its own.
//
// The array (kScratchBytes, about 14 MiB) is a file-scope __device__ variable:
// every GPU that loads the library holds one copy until the process exits.  Its
// device address is looked up with cudaGetSymbolAddress the first time a call
// runs in a given CUDA context (with that context's device current) and cached
// under the context's unique id, so a call made after cudaDeviceReset, or in a
// context other than the device's primary one, looks the address up again
// rather than reuse one that belonged to a context that is gone.  Make the
// first call in a context before any stream capture.  All calls share the one
// array and it keeps the previous call's contents, so the parts that must start
// at zero are cleared on every call, and calls that overlap on the GPU
// (different streams, or different host threads on one device) race on it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "ug_internal.cuh"

namespace {

constexpr uint32_t kNoAllocMaxAgents = 1u << 18;   // 262,144 agents
constexpr uint32_t kNoAllocMaxBoxes = 1u << 20;    // 1,048,576 grid boxes
constexpr size_t kAlign = 256;
constexpr size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
// entries of the box table at the limits (boxes times their x sub-bins)
constexpr size_t kNoAllocTable = (size_t)kNoAllocMaxBoxes + kNoAllocMaxAgents + (kNoAllocMaxAgents >> 2) + 1;
constexpr size_t kNoAllocTiles = (kNoAllocTable + ug::kScanTile - 1) / ug::kScanTile;
// ctrl | bounds | tile sums | counts | table | geometry | key | rank | tmp.
// Every call clears the control words, the bounds, the tile sums of its own
// scan tiles and the counts of its own table; the rest is written before it is
// read.
constexpr size_t kOffBounds = up(sizeof(ug::Ctrl));
constexpr size_t kOffTiles = kOffBounds + up(4ull * ug::kBoundsWords * ug::kBoundsCopiesSingle);
constexpr size_t kTileBytes = 4ull * ug::kTileSumStride * ug::kTileCopies;   // per scan tile
constexpr size_t kOffCounts = kOffTiles + up(kTileBytes * kNoAllocTiles);
constexpr size_t kOffTable = kOffCounts + up(4ull * kNoAllocTable);
constexpr size_t kOffGeo = kOffTable + up(4ull * (kNoAllocTable + 1));
constexpr size_t kOffKey = kOffGeo + up(sizeof(ug_grid_info));
constexpr size_t kOffRank = kOffKey + up(4ull * kNoAllocMaxAgents);
constexpr size_t kOffTmp = kOffRank + up(4ull * kNoAllocMaxAgents);
constexpr size_t kScratchBytes = kOffTmp + up(4ull * kNoAllocMaxAgents);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// cuCtxGetCurrent and cuCtxGetId, fetched through the runtime so that the
// library needs no link against the driver library.
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

std::mutex g_mu;
struct CachedAddress {
    unsigned long long ctx_id;   // 0: empty
    void *addr;
};
CachedAddress g_cache[64] = {};   // one entry per device ordinal

// Unique id of the context current on this thread (0 if it cannot be had).
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
                cudaSuccess && q1 == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
                cudaSuccess && q2 == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f2);
        looked_up = true;
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array in the current context (looked up once
// per context).
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return UG_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = current_context_id();
    if (id == 0) {
        // no context current yet on this thread: make the device's primary
        // context current (cudaSetDevice initialises it), then ask again
        if (cudaSetDevice(dev) != cudaSuccess) return UG_ECUDA;
        id = current_context_id();
        if (id == 0) return UG_ECUDA;
    }
    CachedAddress &c = g_cache[dev];
    if (c.ctx_id != id || c.addr == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
            return UG_ECUDA;
        c.ctx_id = id;
        c.addr = p;
    }
    *out = c.addr;
    return UG_OK;
}

}  // namespace

using namespace ug;

extern "C" int ug_grid_build_noalloc(const float *state_in, const uint32_t *perm_in, uint32_t n,
                                     float contact_margin, float *state_sorted,
                                     uint32_t *perm_sorted, uint32_t *box_start,
                                     uint32_t max_boxes, ug_grid_info *info, int32_t *status,
                                     void *stream) {
    if (n == 0) return UG_OK;
    // the same argument checks as ug_grid_build, then the scratch limits
    auto al = [](const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; };
    if (n > kMaxAgents || !state_in || !al(state_in, 16) || !state_sorted || !al(state_sorted, 16) ||
        !perm_sorted || !box_start || !al(box_start, 16) || !info || !status || max_boxes < 27 ||
        max_boxes > 0x7fffff00u || !(contact_margin >= 0.0f))
        return UG_EINVAL;
    if (n > kNoAllocMaxAgents || max_boxes > kNoAllocMaxBoxes) return UG_EWORKSPACE;
    void *base = nullptr;
    const int rc = scratch_address(&base);
    if (rc != UG_OK) return rc;
    char *b = static_cast<char *>(base);
    Workspace w{};
    w.ctrl = reinterpret_cast<Ctrl *>(b);
    w.counts = reinterpret_cast<uint32_t *>(b + kOffCounts);
    w.bounds = reinterpret_cast<uint32_t *>(b + kOffBounds);
    w.start = reinterpret_cast<uint32_t *>(b + kOffTable);
    w.geo = reinterpret_cast<ug_grid_info *>(b + kOffGeo);
    w.key = reinterpret_cast<uint32_t *>(b + kOffKey);
    w.rank = reinterpret_cast<uint32_t *>(b + kOffRank);
    w.tmp = reinterpret_cast<uint32_t *>(b + kOffTmp);
    w.tile_sum = reinterpret_cast<uint32_t *>(b + kOffTiles);
    const size_t table = (size_t)table_capacity(n, max_boxes);
    w.ntiles = (uint32_t)((table + kScanTile - 1) / kScanTile);
    w.bytes = kScratchBytes;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // tile sums and counts must start at zero; the previous call left them zero
    // unless it failed part-way, so clear them (as far as this call uses them)
    // with the control words and the bounds
    if (cudaMemsetAsync(b, 0, kOffTiles + kTileBytes * w.ntiles, s) != cudaSuccess ||
        cudaMemsetAsync(b + kOffCounts, 0, 4ull * table, s) != cudaSuccess)
        return UG_ECUDA;
    SimArgs sa{};
    sa.nsims = 1;
    sa.n = n;
    sa.pval.contact_margin = contact_margin;
    sa.bounds_copies = kBoundsCopiesSingle;
    const float4 *in = reinterpret_cast<const float4 *>(state_in);
    launch_bounds(in, sa, w, w.geo, max_boxes, status, s);
    launch_key(in, sa, w, w.geo, nullptr, status, s);
    launch_scan(w, w.start, max_boxes, status, s);
    launch_place(w, w.start, n, status, s);
    launch_canon(w, w.start, in, perm_in, reinterpret_cast<float4 *>(state_sorted), perm_sorted,
                 nullptr, n, status, s);
    launch_box_table(w.start, w.geo, box_start, info, max_boxes, status, s);
    return cudaGetLastError() == cudaSuccess ? UG_OK : UG_ECUDA;
}
