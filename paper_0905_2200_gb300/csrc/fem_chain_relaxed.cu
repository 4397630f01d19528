// fem_chain_relaxed.cu -- the relaxed pass (Algorithm 3) in latest-chain form, every length.
#include "fem_chain_launch.cuh"

namespace fem {

cudaError_t launch_chain_relaxed(int N, bool mc, const CountParams &p, uint32_t threads,
                                 cudaStream_t st) {
    return chain_detail::dispatch<FEM_PASS_RELAXED>(N, mc, p, threads, st);
}

size_t chain_smem_bytes(int N, bool mc, uint32_t threads, uint32_t offs) {
    size_t b = 2 * (size_t)stage_bytes(offs) + 128;
    switch (N) {
#define FEM_CASE(n) \
    case n: return b + (mc ? ChainLayout<n, true>::bytes(threads) : ChainLayout<n, false>::bytes(threads));
        FEM_CASE(2) FEM_CASE(3) FEM_CASE(4) FEM_CASE(5) FEM_CASE(6) FEM_CASE(7) FEM_CASE(8)
#undef FEM_CASE
        default: return 0;
    }
}

cudaError_t launch_chain(int N, int pass, bool mc, uint32_t threads, const CountParams &p,
                         cudaStream_t st) {
    if (p.m == 0) return cudaSuccess;
    return pass == FEM_PASS_RELAXED ? launch_chain_relaxed(N, mc, p, threads, st)
                                    : launch_chain_exact(N, mc, p, threads, st);
}

}  // namespace fem
