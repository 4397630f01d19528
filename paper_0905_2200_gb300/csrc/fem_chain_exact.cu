// fem_chain_exact.cu -- the exact pass (Algorithm 1) in latest-chain form, every length.
#include "fem_chain_launch.cuh"

namespace fem {

cudaError_t launch_chain_exact(int N, bool mc, const CountParams &p, uint32_t threads,
                               cudaStream_t st) {
    return chain_detail::dispatch<FEM_PASS_EXACT>(N, mc, p, threads, st);
}

}  // namespace fem
