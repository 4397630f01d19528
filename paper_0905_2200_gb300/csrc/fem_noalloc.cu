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
// fetched with cudaGetSymbolAddress, with the device current, once per device and
// CUDA context (a context created after cudaDeviceReset gets its own lookup).
#include <cuda.h>

#include <mutex>

#include "fem_internal.cuh"

namespace {

// partial sums of one call at the largest size: sized from the compaction's own block
// size (fem_internal.cuh), so a change there resizes the array with it
constexpr size_t kScratchWords = fem::compact_scratch_words_for(FEM_SELECT_NOALLOC_MAX);
static __device__ __align__(256) uint32_t g_select_scratch[kScratchWords];
static_assert(kScratchWords * 4 <= 512 * 1024, "scratch array stays modest");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// per device: the context the address was looked up in (its unique id) and the address
unsigned long long g_ctx_id[kMaxDevices] = {};
uint32_t *g_addr[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context, or 0 if it cannot be had.
// A new context (after cudaDeviceReset, or a non-primary one) gets a new id, so an
// address looked up in another context is never reused.
unsigned long long current_context_id() {
    static decltype(&cuCtxGetCurrent) get_current = nullptr;
    static decltype(&cuCtxGetId) get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        resolved = true;
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                             &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
                cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<decltype(&cuCtxGetCurrent)>(f1);
            get_id = reinterpret_cast<decltype(&cuCtxGetId)>(f2);
        } else {
            cudaGetLastError();
        }
    }
    CUcontext cx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&cx) != CUDA_SUCCESS || !cx ||
        get_id(cx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_select_scratch on `dev` (the current device), looked up once
// per (device, context).
int scratch_address(int dev, uint32_t **out) {
    if (dev < 0 || dev >= kMaxDevices) return FEM_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long id = current_context_id();
    if (!g_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_select_scratch) != cudaSuccess) {
            cudaGetLastError();
            g_addr[dev] = nullptr;
            return FEM_ECUDA;
        }
        g_addr[dev] = static_cast<uint32_t *>(p);
        g_ctx_id[dev] = id;
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
