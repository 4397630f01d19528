// fem_count_exact.cu -- dispatch of the exact pass's counting kernels (Algorithm 1);
// their instantiations are split by episode length over fem_count_exact_n*.cu, which
// compile in parallel.
#include "fem_count_launch.cuh"

namespace fem {

cudaError_t launch_count_exact(int N, bool mc, uint32_t R, const CountParams &p, uint32_t threads,
                               cudaStream_t st, uint32_t classes) {
    switch (N) {
        case 1: case 2: return launch_count_exact_n12(N, mc, R, p, threads, st, classes);
        case 3: case 4: return launch_count_exact_n34(N, mc, R, p, threads, st, classes);
        case 5: case 6: return launch_count_exact_n56(N, mc, R, p, threads, st, classes);
        case 7: case 8: return launch_count_exact_n78(N, mc, R, p, threads, st, classes);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_count_batch_exact(int N, uint32_t R, const launch_detail::BatchArgs &a,
                                     uint32_t threads, int sm_count, cudaStream_t st) {
    switch (N) {
        case 1: case 2: return launch_count_batch_exact_n12(N, R, a, threads, sm_count, st);
        case 3: case 4: return launch_count_batch_exact_n34(N, R, a, threads, sm_count, st);
        case 5: case 6: return launch_count_batch_exact_n56(N, R, a, threads, sm_count, st);
        case 7: case 8: return launch_count_batch_exact_n78(N, R, a, threads, sm_count, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fem
