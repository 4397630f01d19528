// fem_count_relaxed.cu -- the relaxed pass's counting kernels (Algorithm 3), instantiated
// for every episode length.
#include "fem_count_launch.cuh"

namespace fem {

using namespace launch_detail;

cudaError_t launch_count_relaxed(int N, bool mc, const CountParams &p, uint32_t threads,
                              cudaStream_t st, uint32_t classes) {
    switch (N) {
#define FEM_CASE(n)                                                                        \
    case n:                                                                                \
        return mc ? run_r<n, FEM_PASS_RELAXED, true>(1, p, threads, st, classes)        \
                  : run_r<n, FEM_PASS_RELAXED, false>(1, p, threads, st, classes);
        FEM_CASE(1) FEM_CASE(2) FEM_CASE(3) FEM_CASE(4) FEM_CASE(5) FEM_CASE(6) FEM_CASE(7)
        FEM_CASE(8)
#undef FEM_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_count_batch_relaxed(int N, const BatchArgs &a, uint32_t threads,
                                    int sm_count, cudaStream_t st) {
    switch (N) {
#define FEM_CASE(n) \
    case n: return run_batch_r<n, FEM_PASS_RELAXED>(1, a, threads, sm_count, st);
        FEM_CASE(1) FEM_CASE(2) FEM_CASE(3) FEM_CASE(4) FEM_CASE(5) FEM_CASE(6) FEM_CASE(7)
        FEM_CASE(8)
#undef FEM_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fem
