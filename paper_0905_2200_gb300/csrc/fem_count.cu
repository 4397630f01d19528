// fem_count.cu -- instantiation and launch of the counting kernels.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "fem_count.cuh"

namespace fem {

size_t count_smem_bytes(int N, int pass, bool mc, uint32_t ring_cap, uint32_t threads,
                        uint32_t offs) {
    size_t b = 2 * (size_t)stage_bytes(offs) + 128;
    if (pass == FEM_PASS_EXACT && N > 1)
        b += (size_t)(N - 1) * ring_cap * threads * 8u;
    if (mc && N >= 3) b += (size_t)S_MAX * threads * 4u;  // class keys
    return b;
}

bool count_config_supported(int N, int pass, bool mc, uint32_t ring_cap) {
    if (N < 1 || N > FEM_MAX_LEN) return false;
    if (pass == FEM_PASS_RELAXED) return true;
    if (mc) return ring_cap == 8 || ring_cap == 16 || ring_cap == 32;
    return ring_cap == 8 || ring_cap == 16 || ring_cap == 32 || ring_cap == 128;
}

namespace {

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

template <int N, int PASS, bool MC, int R>
cudaError_t run(const CountParams &p, uint32_t threads, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(count_kernel<N, PASS, MC, R>(),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const size_t sm = count_smem_bytes(N, PASS, MC, R, threads, p.offs);
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    dim3 grid((p.m + threads - 1) / threads, p.P);
    count_kernel<N, PASS, MC, R>()<<<grid, threads, sm, st>>>(p);
    note_launch();
    return cudaGetLastError();
}

template <int N, int PASS, bool MC>
cudaError_t run_r(uint32_t R, const CountParams &p, uint32_t threads, cudaStream_t st) {
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

template <int N>
cudaError_t run_n(int pass, bool mc, uint32_t R, const CountParams &p, uint32_t threads,
                  cudaStream_t st) {
    if (pass == FEM_PASS_RELAXED)
        return mc ? run_r<N, FEM_PASS_RELAXED, true>(R, p, threads, st)
                  : run_r<N, FEM_PASS_RELAXED, false>(R, p, threads, st);
    return mc ? run_r<N, FEM_PASS_EXACT, true>(R, p, threads, st)
              : run_r<N, FEM_PASS_EXACT, false>(R, p, threads, st);
}

template <int N>
cudaError_t run_batch_n(int pass, uint32_t R, const BatchArgs &a, uint32_t threads, int sm_count,
                        cudaStream_t st) {
    return pass == FEM_PASS_RELAXED
               ? run_batch_r<N, FEM_PASS_RELAXED>(R, a, threads, sm_count, st)
               : run_batch_r<N, FEM_PASS_EXACT>(R, a, threads, sm_count, st);
}

}  // namespace

cudaError_t launch_count_batch(int N, int pass, uint32_t ring_cap, uint32_t threads,
                               const CountParams *jobs, const uint4 *items,
                               const uint32_t *n_items, uint32_t *queue, uint32_t SB,
                               int sm_count, cudaStream_t st) {
    const BatchArgs a{jobs, items, n_items, queue, SB, 0};
    switch (N) {
        case 1: return run_batch_n<1>(pass, ring_cap, a, threads, sm_count, st);
        case 2: return run_batch_n<2>(pass, ring_cap, a, threads, sm_count, st);
        case 3: return run_batch_n<3>(pass, ring_cap, a, threads, sm_count, st);
        case 4: return run_batch_n<4>(pass, ring_cap, a, threads, sm_count, st);
        case 5: return run_batch_n<5>(pass, ring_cap, a, threads, sm_count, st);
        case 6: return run_batch_n<6>(pass, ring_cap, a, threads, sm_count, st);
        case 7: return run_batch_n<7>(pass, ring_cap, a, threads, sm_count, st);
        case 8: return run_batch_n<8>(pass, ring_cap, a, threads, sm_count, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_count(int N, int pass, bool mc, uint32_t ring_cap, uint32_t threads,
                         const CountParams &p, cudaStream_t st) {
    if (p.m == 0) return cudaSuccess;
    switch (N) {
        case 1: return run_n<1>(pass, mc, ring_cap, p, threads, st);
        case 2: return run_n<2>(pass, mc, ring_cap, p, threads, st);
        case 3: return run_n<3>(pass, mc, ring_cap, p, threads, st);
        case 4: return run_n<4>(pass, mc, ring_cap, p, threads, st);
        case 5: return run_n<5>(pass, mc, ring_cap, p, threads, st);
        case 6: return run_n<6>(pass, mc, ring_cap, p, threads, st);
        case 7: return run_n<7>(pass, mc, ring_cap, p, threads, st);
        case 8: return run_n<8>(pass, mc, ring_cap, p, threads, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fem
