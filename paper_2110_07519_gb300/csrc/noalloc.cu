// noalloc.cu -- messi_lower_bounds_noalloc: the per-series lower bounds of
// one query against an existing index, computed without allocating memory.
//
// Who needs it: callers that may not call cudaMalloc while they run -- an
// embedding that owns a fixed device-memory budget and hands the library
// only its input and output buffers, or a latency-critical loop that must
// not stall in the allocator (cudaMalloc and cudaFree can synchronise the
// device and wait for other streams' work).  messi_lower_bounds() keeps its
// scratch (query state, the lower-bound table, the query and its envelope)
// in a workspace it allocates on first use; this entry point keeps the same
// scratch in the fixed-size file-scope array below instead, which every GPU
// that loads the library holds until the process exits.
#include <mutex>
#include <vector>

#include "messi_internal.cuh"

namespace messi {
namespace {

// Maximum series length this entry point accepts: the query and its two
// envelope rows (3 x 2048 floats) plus the 16 x 256 table and the query state.
constexpr int kNoAllocMaxLen = 2048;
constexpr size_t kStateBytes = 256;
constexpr size_t kLutBytes = kMaxSegments * kMaxCard * 4;
constexpr size_t kRowBytes = kNoAllocMaxLen * 4;
constexpr size_t kScratchBytes = kStateBytes + kLutBytes + 3 * kRowBytes;   // 40,960 + 256 bytes
static_assert(sizeof(QueryState) <= kStateBytes, "query state must fit its scratch slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array, looked up once per device with that
// device current.  In host code the array's name is only a host-side stand-in.
std::mutex g_mu;
std::vector<void *> g_addr;   // indexed by device ordinal

messi_status scratch_address(int dev, void **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_addr.size() <= dev) g_addr.resize(dev + 1, nullptr);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (!cuda_ok(cudaGetSymbolAddress(&p, g_noalloc_scratch), "messi_lower_bounds_noalloc: cudaGetSymbolAddress"))
            return MESSI_ECUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return MESSI_OK;
}

}  // namespace
}  // namespace messi

using namespace messi;

extern "C" messi_status messi_lower_bounds_noalloc(const messi_index *ix, const float *query, messi_dist dist,
                                                   uint32_t window, float *lb2, messi_stream stream)
{
    if (!ix || !query || !lb2) return fail(MESSI_EINVAL, "messi_lower_bounds_noalloc: null argument");
    if (dist != MESSI_ED && dist != MESSI_DTW)
        return fail(MESSI_EINVAL, "messi_lower_bounds_noalloc: unknown distance");
    if (dist == MESSI_DTW && window >= (uint32_t)ix->len)
        return fail(MESSI_EINVAL, "messi_lower_bounds_noalloc: window must be < len");
    if (ix->len > kNoAllocMaxLen)
        return fail(MESSI_EINVAL, "messi_lower_bounds_noalloc: series length exceeds the 2048-point maximum "
                                  "of its fixed scratch; use messi_lower_bounds");
    if (!is_device_ptr(query) || !is_device_ptr(lb2))
        return fail(MESSI_EINVAL, "messi_lower_bounds_noalloc: query and lb2 must be device pointers "
                                  "(host buffers would need staging memory)");
    // the index, both buffers and the scratch used below must all be the
    // current device's memory
    const void *ptrs[2] = {query, lb2};
    messi_status st = check_device(ix, ptrs, 2, "messi_lower_bounds_noalloc");
    if (st != MESSI_OK) return st;
    void *base = nullptr;
    if ((st = scratch_address(ix->device, &base)) != MESSI_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *b = static_cast<char *>(base);

    QuerySlot slot{};
    slot.st = reinterpret_cast<QueryState *>(b);
    slot.lut = reinterpret_cast<float *>(b + kStateBytes);
    slot.q = reinterpret_cast<float *>(b + kStateBytes + kLutBytes);
    slot.U = reinterpret_cast<float *>(b + kStateBytes + kLutBytes + kRowBytes);
    slot.L = reinterpret_cast<float *>(b + kStateBytes + kLutBytes + 2 * kRowBytes);
    slot.log_cap = 0;   // no candidates are logged on this path
    // the array keeps the previous call's contents: the query state starts at zero
    if (!cuda_ok(cudaMemsetAsync(slot.st, 0, kStateBytes, s), "messi_lower_bounds_noalloc: clear state"))
        return MESSI_ECUDA;

    const IndexView iv = view_of(ix);
    const QueryParams qp = make_params(ix, 1, (int)dist, window);
    launch_prep(iv, qp, slot, query, s);
    launch_lower_bounds(iv, slot, lb2, s);
    if (!cuda_ok(cudaGetLastError(), "messi_lower_bounds_noalloc: launch")) return MESSI_ECUDA;
    return MESSI_OK;
}
