// fem_noalloc.cu -- fem_select_noalloc: the survivor selection of the two-pass count
// for callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a
// real-time acquisition loop that owns a fixed, pre-reserved memory budget, or in
// a host thread that must never trigger the implicit device synchronisation of
// cudaMalloc/cudaFree.  Such a caller already holds its inputs and outputs on the
// device and only needs the per-block partial sums of the compaction somewhere.
//
// Those partial sums live in a file-scope device array of fixed size.  Every GPU
// that loads this library holds the array (about 256 KB) until the process exits.
// Host code cannot use the array's name as a device address: the address is
// fetched once per device with cudaGetSymbolAddress, with that device current.
#include <mutex>

#include "fem_internal.cuh"

namespace {

constexpr uint32_t kItemsPerBlock = 1024;  // items one compaction block handles
constexpr uint32_t kMaxBlocks = FEM_SELECT_NOALLOC_MAX / kItemsPerBlock;

// per-block partial sums of one call, plus the slack launch_compact expects
static __device__ __align__(256) uint32_t g_select_scratch[kMaxBlocks + 32];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t *g_addr[kMaxDevices] = {};

// Device address of g_select_scratch on `dev` (the current device).
int scratch_address(int dev, uint32_t **out) {
    if (dev < 0 || dev >= kMaxDevices) return FEM_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_select_scratch) != cudaSuccess) {
            cudaGetLastError();
            return FEM_ECUDA;
        }
        g_addr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_addr[dev];
    return FEM_OK;
}

}  // namespace

extern "C" int fem_select_noalloc(const uint32_t *values, uint32_t m, uint32_t theta,
                                  uint32_t *idx_out, uint32_t *count_out, void *cuda_stream) {
    if (!count_out || (m && (!values || !idx_out))) return FEM_EINVAL;
    if (m > FEM_SELECT_NOALLOC_MAX) return FEM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return FEM_ECUDA;
    }
    uint32_t *scratch = nullptr;
    const int rc = scratch_address(dev, &scratch);
    if (rc != FEM_OK) return rc;
    // every partial sum the three kernels read is written earlier in the same call,
    // so nothing needs clearing between calls
    if (fem::launch_compact(values, nullptr, theta, m, idx_out, count_out, scratch,
                            static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess) {
        cudaGetLastError();
        return FEM_ECUDA;
    }
    return FEM_OK;
}
