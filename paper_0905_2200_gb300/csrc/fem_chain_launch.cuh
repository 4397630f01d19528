// fem_chain_launch.cuh -- launch template of the latest-chain counting kernels,
// instantiated per pass in fem_chain_relaxed.cu and fem_chain_exact.cu.
#pragma once

#include <mutex>

#include "fem_chain.cuh"

namespace fem {
namespace chain_detail {

template <int N, int PASS, bool MC>
cudaError_t run(const CountParams &p, uint32_t threads, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(k_chain<N, PASS, MC>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    if (attr_err != cudaSuccess) return attr_err;
    if (threads < 32 || threads > 256 || threads % 32) return cudaErrorInvalidConfiguration;
    const size_t sm = 2 * (size_t)stage_bytes(p.offs) + 128 + ChainLayout<N, MC>::bytes(threads);
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    dim3 grid((p.m + threads - 1) / threads, p.P);
    k_chain<N, PASS, MC><<<grid, threads, sm, st>>>(p);
    note_launch();
    return cudaGetLastError();
}

template <int PASS>
cudaError_t dispatch(int N, bool mc, const CountParams &p, uint32_t threads, cudaStream_t st) {
    switch (N) {
#define FEM_CASE(n) \
    case n: return mc ? run<n, PASS, true>(p, threads, st) : run<n, PASS, false>(p, threads, st);
        FEM_CASE(2) FEM_CASE(3) FEM_CASE(4) FEM_CASE(5) FEM_CASE(6) FEM_CASE(7) FEM_CASE(8)
#undef FEM_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace chain_detail

cudaError_t launch_chain_relaxed(int N, bool mc, const CountParams &p, uint32_t threads,
                                 cudaStream_t st);
cudaError_t launch_chain_exact(int N, bool mc, const CountParams &p, uint32_t threads,
                               cudaStream_t st);

}  // namespace fem
