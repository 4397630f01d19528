// fem_count_exact_n56.cu -- the exact pass's counting kernels for episodes of 5
// and 6 nodes.
#include "fem_count_launch.cuh"

namespace fem {

using namespace launch_detail;

cudaError_t launch_count_exact_n56(int N, bool mc, uint32_t R, const CountParams &p,
                                  uint32_t threads, cudaStream_t st, uint32_t classes) {
    if (N == 5)
        return mc ? run_r<5, FEM_PASS_EXACT, true>(R, p, threads, st, classes)
                  : run_r<5, FEM_PASS_EXACT, false>(R, p, threads, st, classes);
    if (N == 6)
        return mc ? run_r<6, FEM_PASS_EXACT, true>(R, p, threads, st, classes)
                  : run_r<6, FEM_PASS_EXACT, false>(R, p, threads, st, classes);
    return cudaErrorInvalidValue;
}

cudaError_t launch_count_batch_exact_n56(int N, uint32_t R, const BatchArgs &a,
                                        uint32_t threads, int sm_count, cudaStream_t st) {
    if (N == 5) return run_batch_r<5, FEM_PASS_EXACT>(R, a, threads, sm_count, st);
    if (N == 6) return run_batch_r<6, FEM_PASS_EXACT>(R, a, threads, sm_count, st);
    return cudaErrorInvalidValue;
}

}  // namespace fem
