// fem_count_launch.cuh -- launch templates of the counting kernels, instantiated per
// pass in fem_count_relaxed.cu and fem_count_exact.cu (two translation units that
// compile in parallel).
#pragma once

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "fem_count.cuh"

namespace fem {
namespace launch_detail {

struct BatchArgs {
    const CountParams *jobs;
    const uint4 *items;
    const uint32_t *n_items;
    uint32_t *queue;
    uint32_t SB;
    uint32_t blocks;  // 0: one wave of resident blocks
};

template <int N, int PASS, bool MC, int R>
cudaError_t run_batch(const BatchArgs &a, uint32_t threads, int sm_count, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(count_batch_kernel<N, PASS, MC, R>(),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    if (attr_err != cudaSuccess) return attr_err;
    size_t sm = 2 * (size_t)a.SB + 128 + (N >= 3 ? (size_t)S_MAX * threads * 4u : 0);  // keys
    if (PASS == FEM_PASS_EXACT && N > 1) sm += (size_t)(N - 1) * R * threads * 8u;
    if (sm > 200 * 1024) return cudaErrorInvalidConfiguration;
    uint32_t blocks = a.blocks;
    if (!blocks) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, count_batch_kernel<N, PASS, MC, R>(), (int)threads, sm);
        if (e != cudaSuccess) return e;
        blocks = (uint32_t)std::max(1, per_sm) * (uint32_t)sm_count;
    }
    count_batch_kernel<N, PASS, MC, R>()<<<blocks, threads, sm, st>>>(a.jobs, a.items, a.n_items,
                                                               a.queue, a.SB);
    note_launch();
    return cudaGetLastError();
}

template <int N, int PASS>
cudaError_t run_batch_r(uint32_t R, const BatchArgs &a, uint32_t threads, int sm_count,
                        cudaStream_t st) {
    if constexpr (PASS == FEM_PASS_RELAXED) {
        return run_batch<N, PASS, true, 1>(a, threads, sm_count, st);
    } else {
        switch (R) {
            case 8: return run_batch<N, PASS, true, 8>(a, threads, sm_count, st);
            case 16: return run_batch<N, PASS, true, 16>(a, threads, sm_count, st);
            case 32: return run_batch<N, PASS, true, 32>(a, threads, sm_count, st);
            default: return cudaErrorInvalidValue;
        }
    }
}

template <int N, int PASS, bool MC, int R, int SMX = S_MAX>
cudaError_t run(const CountParams &p, uint32_t threads, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(count_kernel<N, PASS, MC, R, SMX>(),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const size_t sm = count_smem_bytes(N, PASS, MC, R, threads, p.offs, SMX);
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    dim3 grid((p.m + threads - 1) / threads, p.P);
    count_kernel<N, PASS, MC, R, SMX>()<<<grid, threads, sm, st>>>(p);
    note_launch();
    return cudaGetLastError();
}

// classes = 16: the recount's segmented form (relaxed, or exact with rings of 32)
template <int N, int PASS, bool MC>
cudaError_t run_r(uint32_t R, const CountParams &p, uint32_t threads, cudaStream_t st,
                  uint32_t classes) {
    if (classes == S_RECOUNT) {
        if constexpr (MC) {
            if constexpr (PASS == FEM_PASS_RELAXED) return run<N, PASS, MC, 1, S_RECOUNT>(p, threads, st);
            else if (R == 32) return run<N, PASS, MC, 32, S_RECOUNT>(p, threads, st);
        }
        return cudaErrorInvalidValue;
    }
    if constexpr (PASS == FEM_PASS_RELAXED) {
        return run<N, PASS, MC, 1>(p, threads, st);
    } else {
        switch (R) {
            case 8: return run<N, PASS, MC, 8>(p, threads, st);
            case 16: return run<N, PASS, MC, 16>(p, threads, st);
            case 32: return run<N, PASS, MC, 32>(p, threads, st);
            case 128:
                if constexpr (!MC) return run<N, PASS, MC, 128>(p, threads, st);
                else return cudaErrorInvalidValue;
            default: return cudaErrorInvalidValue;
        }
    }
}

}  // namespace launch_detail

// per-pass entry points (one translation unit each)
cudaError_t launch_count_relaxed(int N, bool mc, const CountParams &p, uint32_t threads,
                                 cudaStream_t st, uint32_t classes);
cudaError_t launch_count_exact(int N, bool mc, uint32_t R, const CountParams &p, uint32_t threads,
                               cudaStream_t st, uint32_t classes);
cudaError_t launch_count_batch_relaxed(int N, const launch_detail::BatchArgs &a, uint32_t threads,
                                       int sm_count, cudaStream_t st);
cudaError_t launch_count_batch_exact(int N, uint32_t R, const launch_detail::BatchArgs &a,
                                     uint32_t threads, int sm_count, cudaStream_t st);
#define FEM_EXACT_RANGE(ab)                                                                    \
    cudaError_t launch_count_exact_n##ab(int N, bool mc, uint32_t R, const CountParams &p,      \
                                         uint32_t threads, cudaStream_t st, uint32_t classes); \
    cudaError_t launch_count_batch_exact_n##ab(int N, uint32_t R, const launch_detail::BatchArgs &a, \
                                               uint32_t threads, int sm_count, cudaStream_t st);
FEM_EXACT_RANGE(12)
FEM_EXACT_RANGE(34)
FEM_EXACT_RANGE(56)
FEM_EXACT_RANGE(78)
#undef FEM_EXACT_RANGE

}  // namespace fem
