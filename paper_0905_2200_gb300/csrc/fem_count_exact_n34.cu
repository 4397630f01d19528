// fem_count_exact_n34.cu -- the exact pass's counting kernels for episodes of 3
// and 4 nodes.
#include "fem_count_launch.cuh"

namespace fem {

using namespace launch_detail;

cudaError_t launch_count_exact_n34(int N, bool mc, uint32_t R, const CountParams &p,
                                  uint32_t threads, cudaStream_t st, uint32_t classes) {
    if (N == 3)
        return mc ? run_r<3, FEM_PASS_EXACT, true>(R, p, threads, st, classes)
                  : run_r<3, FEM_PASS_EXACT, false>(R, p, threads, st, classes);
    if (N == 4)
        return mc ? run_r<4, FEM_PASS_EXACT, true>(R, p, threads, st, classes)
                  : run_r<4, FEM_PASS_EXACT, false>(R, p, threads, st, classes);
    return cudaErrorInvalidValue;
}

cudaError_t launch_count_batch_exact_n34(int N, uint32_t R, const BatchArgs &a,
                                        uint32_t threads, int sm_count, cudaStream_t st) {
    if (N == 3) return run_batch_r<3, FEM_PASS_EXACT>(R, a, threads, sm_count, st);
    if (N == 4) return run_batch_r<4, FEM_PASS_EXACT>(R, a, threads, sm_count, st);
    return cudaErrorInvalidValue;
}

}  // namespace fem
