// fem_count.cu -- shared-memory sizing and the pass dispatch of the counting kernels
// (their instantiations live in fem_count_relaxed.cu and fem_count_exact.cu).
#include "fem_count_launch.cuh"

namespace fem {

size_t count_smem_bytes(int N, int pass, bool mc, uint32_t ring_cap, uint32_t threads,
                        uint32_t offs, uint32_t classes) {
    size_t b = 2 * (size_t)stage_bytes(offs) + 128;
    if (pass == FEM_PASS_EXACT && N > 1)
        b += (size_t)(N - 1) * ring_cap * threads * 8u;
    if (mc && N >= 3) b += (size_t)classes * threads * 4u;  // class keys
    return b;
}

bool count_config_supported(int N, int pass, bool mc, uint32_t ring_cap) {
    if (N < 1 || N > FEM_MAX_LEN) return false;
    if (pass == FEM_PASS_RELAXED) return true;
    if (mc) return ring_cap == 8 || ring_cap == 16 || ring_cap == 32;
    return ring_cap == 8 || ring_cap == 16 || ring_cap == 32 || ring_cap == 128;
}

cudaError_t launch_count_batch(int N, int pass, uint32_t ring_cap, uint32_t threads,
                               const CountParams *jobs, const uint4 *items,
                               const uint32_t *n_items, uint32_t *queue, uint32_t SB,
                               int sm_count, cudaStream_t st) {
    const launch_detail::BatchArgs a{jobs, items, n_items, queue, SB, 0};
    return pass == FEM_PASS_RELAXED ? launch_count_batch_relaxed(N, a, threads, sm_count, st)
                                    : launch_count_batch_exact(N, ring_cap, a, threads, sm_count, st);
}

cudaError_t launch_count(int N, int pass, bool mc, uint32_t ring_cap, uint32_t threads,
                         const CountParams &p, cudaStream_t st, uint32_t classes) {
    if (p.m == 0) return cudaSuccess;
    return pass == FEM_PASS_RELAXED ? launch_count_relaxed(N, mc, p, threads, st, classes)
                                    : launch_count_exact(N, mc, ring_cap, p, threads, st, classes);
}

}  // namespace fem
