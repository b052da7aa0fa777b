// Grid build that allocates nothing: its scratch space is a fixed array of
// device memory compiled into the library, for callers that cannot allocate.
//
// Who needs it: a caller that is handed only its inputs and outputs and may not
// allocate device memory at the point of the call -- for instance a plug-in
// whose host application owns every byte of the GPU's memory, or code that runs
// under a fixed memory budget.  Such a caller cannot supply the workspace that
// ug_grid_build asks for, so this variant brings its own.
//
// The array (kScratchBytes, about 7 MiB) is a file-scope __device__ variable:
// every GPU that loads the library holds one copy until the process exits.  The
// first call on a device looks up the array's device address with
// cudaGetSymbolAddress (once per device, with that device current); make that
// first call before any stream capture.  All calls share the one array and it
// keeps the previous call's contents, so the parts that must start at zero are
// cleared on every call, and calls that overlap on the GPU (different streams,
// or different host threads on one device) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "ug_internal.cuh"

namespace {

constexpr uint32_t kNoAllocMaxAgents = 1u << 18;   // 262,144 agents
constexpr uint32_t kNoAllocMaxBoxes = 1u << 20;    // 1,048,576 grid boxes
constexpr size_t kAlign = 256;
constexpr size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kNoAllocTiles = (kNoAllocMaxBoxes + ug::kScanTile - 1) / ug::kScanTile;
// ctrl | tile sums | counts | bounds (these four are zeroed per call) | key | rank | tmp
constexpr size_t kOffTiles = up(sizeof(ug::Ctrl));
constexpr size_t kOffCounts = kOffTiles + up(4ull * ug::kTileSumStride * ug::kTileCopies * kNoAllocTiles);
constexpr size_t kOffBounds = kOffCounts + up(4ull * kNoAllocMaxBoxes);
constexpr size_t kOffKey = kOffBounds + up(4ull * ug::kBoundsWords * ug::kBoundsCopiesSingle);
constexpr size_t kOffRank = kOffKey + up(4ull * kNoAllocMaxAgents);
constexpr size_t kOffTmp = kOffRank + up(4ull * kNoAllocMaxAgents);
constexpr size_t kScratchBytes = kOffTmp + up(4ull * kNoAllocMaxAgents);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return UG_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
            return UG_ECUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
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
    if (n > kNoAllocMaxAgents || max_boxes > kNoAllocMaxBoxes) return UG_EWORKSPACE;
    auto al = [](const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; };
    if (!state_in || !al(state_in, 16) || !state_sorted || !al(state_sorted, 16) || !perm_sorted ||
        !box_start || !al(box_start, 16) || !info || !status || max_boxes < 27 ||
        !(contact_margin >= 0.0f))
        return UG_EINVAL;
    void *base = nullptr;
    const int rc = scratch_address(&base);
    if (rc != UG_OK) return rc;
    char *b = static_cast<char *>(base);
    Workspace w{};
    w.ctrl = reinterpret_cast<Ctrl *>(b);
    w.counts = reinterpret_cast<uint32_t *>(b + kOffCounts);
    w.bounds = reinterpret_cast<uint32_t *>(b + kOffBounds);
    w.key = reinterpret_cast<uint32_t *>(b + kOffKey);
    w.rank = reinterpret_cast<uint32_t *>(b + kOffRank);
    w.tmp = reinterpret_cast<uint32_t *>(b + kOffTmp);
    w.tile_sum = reinterpret_cast<uint32_t *>(b + kOffTiles);
    w.ntiles = (max_boxes + kScanTile - 1) / kScanTile;
    w.bytes = kScratchBytes;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // tile sums and counts must start at zero; the previous call left them zero
    // unless it failed part-way, so clear them with the control words and bounds
    if (cudaMemsetAsync(b, 0, kOffBounds + 4ull * kBoundsWords * kBoundsCopiesSingle, s) != cudaSuccess)
        return UG_ECUDA;
    SimArgs sa{};
    sa.nsims = 1;
    sa.n = n;
    sa.pval.contact_margin = contact_margin;
    sa.bounds_copies = kBoundsCopiesSingle;
    const float4 *in = reinterpret_cast<const float4 *>(state_in);
    launch_bounds(in, sa, w, info, max_boxes, status, s);
    launch_key(in, sa, w, info, nullptr, status, s);
    launch_scan(w, box_start, max_boxes, status, s);
    launch_place(w, box_start, n, status, s);
    launch_canon(w, box_start, in, perm_in, reinterpret_cast<float4 *>(state_sorted), perm_sorted,
                 nullptr, n, status, s);
    return cudaGetLastError() == cudaSuccess ? UG_OK : UG_ECUDA;
}
