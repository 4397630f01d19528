// fem_batch.cu -- device-side bookkeeping of a batch of counting jobs (many
// recordings, each with its own candidate set of one episode length), so that a
// whole two-pass count of the batch runs without a host round trip and can be
// captured once in a CUDA graph:
//   work items (job, episode tile, segment) built from device-resident job sizes,
//   per-job thresholds for Algorithm 4's elimination, per-job survivor ranges
//   after the (global, stable) compaction, and the scatter of exact counts into
//   each job's own output arrays.
#include <algorithm>

#include "fem_internal.cuh"

namespace fem {

namespace {

// last j in [0, n) with base[j] <= x (base ascending, base[0] <= x)
__device__ __forceinline__ uint32_t find_job(const uint32_t *base, uint32_t n, uint32_t x) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (base[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// first k in [0, cnt) with idx[k] >= x
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *idx, uint32_t cnt, uint32_t x) {
    uint32_t lo = 0, hi = cnt;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (idx[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

}  // namespace

// item_off[j] = items of jobs before j (tiles of T episodes x segments); *n_items = total.
__global__ void __launch_bounds__(1024) k_batch_item_counts(const CountParams *__restrict__ jobs,
                                                             uint32_t n_jobs, uint32_t T,
                                                             uint32_t *__restrict__ item_off,
                                                             uint32_t *__restrict__ n_items) {
    __shared__ uint32_t carry;
    __shared__ uint32_t wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (uint32_t base = 0; base < n_jobs; base += blockDim.x) {
        const uint32_t j = base + threadIdx.x;
        uint32_t v = 0;
        if (j < n_jobs) v = ((jobs[j].m + T - 1) / T) * jobs[j].P;
        uint32_t inc = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= (uint32_t)d) inc += y;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        uint32_t woff = 0;
        for (uint32_t q = 0; q < w; ++q) woff += wsum[q];
        if (j < n_jobs) item_off[j] = carry + woff + inc - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += woff + inc;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        item_off[n_jobs] = carry;
        *n_items = carry;
    }
}

// items[it] = (job, tile, segment) for it < *n_items; segment-major within a job.
__global__ void k_batch_fill_items(const CountParams *__restrict__ jobs, uint32_t n_jobs,
                                   uint32_t T, const uint32_t *__restrict__ item_off,
                                   const uint32_t *__restrict__ n_items, uint32_t cap,
                                   uint4 *__restrict__ items) {
    const uint32_t total = min(*n_items, cap);
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < total;
         it += gridDim.x * blockDim.x) {
        const uint32_t j = find_job(item_off, n_jobs, it);
        const uint32_t r = it - item_off[j];
        const uint32_t tiles = (jobs[j].m + T - 1) / T;
        items[it] = make_uint4(j, r % tiles, r / tiles, 0);
    }
}

cudaError_t launch_batch_items(const CountParams *jobs, uint32_t n_jobs, uint32_t T,
                               uint32_t *item_off, uint32_t *n_items, uint32_t cap, uint4 *items,
                               cudaStream_t st) {
    k_batch_item_counts<<<1, 1024, 0, st>>>(jobs, n_jobs, T, item_off, n_items);
    note_launch();
    const uint32_t blocks = (uint32_t)std::min<uint64_t>((cap + 255) / 256, 4096);
    k_batch_fill_items<<<blocks ? blocks : 1, 256, 0, st>>>(jobs, n_jobs, T, item_off, n_items,
                                                            cap, items);
    note_launch();
    return cudaGetLastError();
}

// flags[i] = rel[i] >= theta of the job candidate i belongs to (cand_off: n_jobs + 1).
__global__ void k_batch_keep_flags(const uint32_t *__restrict__ rel,
                                   const uint32_t *__restrict__ cand_off,
                                   const uint32_t *__restrict__ theta, uint32_t n_jobs,
                                   uint32_t m, uint8_t *__restrict__ flags) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        flags[i] = rel[i] >= theta[find_job(cand_off, n_jobs, i)];
}

cudaError_t launch_batch_keep_flags(const uint32_t *rel, const uint32_t *cand_off,
                                    const uint32_t *theta, uint32_t n_jobs, uint32_t m,
                                    uint8_t *flags, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    const uint32_t blocks = (uint32_t)std::min<uint64_t>((m + 255) / 256, 4096);
    k_batch_keep_flags<<<blocks, 256, 0, st>>>(rel, cand_off, theta, n_jobs, m, flags);
    note_launch();
    return cudaGetLastError();
}

// Exact-pass job j counts the survivors idx[s_j .. e_j) (global candidate indices,
// ascending) of its candidate range [cand_off[j], cand_off[j+1]).
__global__ void k_batch_exact_jobs(CountParams *__restrict__ xjobs,
                                   const uint32_t *__restrict__ cand_off, uint32_t n_jobs,
                                   const uint32_t *__restrict__ idx,
                                   const uint32_t *__restrict__ n_idx, uint32_t *__restrict__ ex) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_jobs) return;
    const uint32_t cnt = *n_idx;
    const uint32_t s = lower_bound_u32(idx, cnt, cand_off[j]);
    const uint32_t e = lower_bound_u32(idx, cnt, cand_off[j + 1]);
    xjobs[j].m = e - s;
    xjobs[j].gather = idx + s;
    xjobs[j].out = ex + s;
}

cudaError_t launch_batch_exact_jobs(CountParams *xjobs, const uint32_t *cand_off, uint32_t n_jobs,
                                    const uint32_t *idx, const uint32_t *n_idx, uint32_t *ex,
                                    cudaStream_t st) {
    k_batch_exact_jobs<<<(n_jobs + 127) / 128, 128, 0, st>>>(xjobs, cand_off, n_jobs, idx, n_idx,
                                                             ex);
    note_launch();
    return cudaGetLastError();
}

// Zero every job's outputs, then write the exact count and survived flag of each
// survivor (idx ascending, ex in the same order).
__global__ void k_batch_zero_out(const BatchOut *__restrict__ outs,
                                 const uint32_t *__restrict__ cand_off, uint32_t n_jobs,
                                 uint32_t m) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const uint32_t j = find_job(cand_off, n_jobs, i);
        const uint32_t r = i - cand_off[j];
        outs[j].exact[r] = 0;
        outs[j].survived[r] = 0;
    }
}

__global__ void k_batch_scatter(const BatchOut *__restrict__ outs,
                                const uint32_t *__restrict__ cand_off, uint32_t n_jobs,
                                const uint32_t *__restrict__ idx,
                                const uint32_t *__restrict__ n_idx,
                                const uint32_t *__restrict__ ex) {
    const uint32_t cnt = *n_idx;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt;
         k += gridDim.x * blockDim.x) {
        const uint32_t c = idx[k];
        const uint32_t j = find_job(cand_off, n_jobs, c);
        const uint32_t r = c - cand_off[j];
        outs[j].exact[r] = ex[k];
        outs[j].survived[r] = 1;
    }
}

cudaError_t launch_batch_outputs(const BatchOut *outs, const uint32_t *cand_off, uint32_t n_jobs,
                                 uint32_t m, const uint32_t *idx, const uint32_t *n_idx,
                                 const uint32_t *ex, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    const uint32_t blocks = (uint32_t)std::min<uint64_t>((m + 255) / 256, 4096);
    k_batch_zero_out<<<blocks, 256, 0, st>>>(outs, cand_off, n_jobs, m);
    note_launch();
    k_batch_scatter<<<blocks, 256, 0, st>>>(outs, cand_off, n_jobs, idx, n_idx, ex);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fem
