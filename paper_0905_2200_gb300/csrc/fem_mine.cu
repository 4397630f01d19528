// fem_mine.cu -- the kernels around the counters: MapConcatenate stitch,
// candidate validation, stable compaction (Algorithm 4's elimination), scans,
// and level-wise candidate generation.
#include <string.h>

#include <algorithm>

#include "fem_internal.cuh"

namespace fem {

namespace {

__device__ __forceinline__ fem_episode ld_ep(const fem_episode *p, uint64_t i) {
    const uint4 v = reinterpret_cast<const uint4 *>(p)[i];
    fem_episode e;
    memcpy(&e, &v, sizeof(e));
    return e;
}
__device__ __forceinline__ void st_ep(fem_episode *p, uint64_t i, const fem_episode &e) {
    uint4 v;
    memcpy(&v, &e, sizeof(v));
    reinterpret_cast<uint4 *>(p)[i] = v;
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024).
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t wtotal;
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= (uint32_t)d) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const uint32_t nw = (blockDim.x + 31) >> 5;
        uint32_t s = lane < nw ? wsum[lane] : 0u;
        uint32_t si = s;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, si, d);
            if (lane >= (uint32_t)d) si += y;
        }
        if (lane < nw) wsum[lane] = si - s;
        if (lane == nw - 1) wtotal = si;
    }
    __syncthreads();
    const uint32_t res = wsum[w] + inc - v;
    if (total) *total = wtotal;
    __syncthreads();
    return res;
}

constexpr uint32_t CT = 256;          // threads per compaction block
constexpr uint32_t CI = 4;            // items per thread
constexpr uint32_t CB = CT * CI;      // items per block
static_assert(CB == COMPACT_ITEMS_PER_BLOCK, "compaction block size is declared in fem_internal.cuh");

__device__ __forceinline__ bool keep_at(const uint32_t *vals, const uint8_t *flags, uint32_t theta,
                                        uint32_t i) {
    return vals ? vals[i] >= theta : flags[i] != 0;
}

}  // namespace

// ------------------------------------------------------------------ MapConcatenate stitch
// stitch_run<SMX, SU>: the composition with tables of SMX slots (the layout) of which
// at most SU can hold a class anywhere in the warp's tables; every loop is unrolled
// and branch-free over SU slots.  G lanes (a power of two) work on one episode; lane
// gl of the group holds segments [a, b); `live` is false for a group past the end of
// the candidates or flagged for a recount (it only takes part in the shuffles).
template <int SMX, int SU>
__device__ __forceinline__ void stitch_run(const uint4 *__restrict__ tables, uint32_t m, uint32_t a,
                                           uint32_t b, uint32_t ci, uint32_t G, uint32_t gl,
                                           bool live, uint32_t *__restrict__ out,
                                           uint8_t *__restrict__ redo, uint32_t *err) {
    const uint32_t lane = threadIdx.x & 31;
    uint32_t fk[SU], fc[SU], fe[SU];
    bool ident = !live || a == b, bad = false;
#pragma unroll
    for (int j = 0; j < SU; ++j) fk[j] = CLS_EMPTY, fc[j] = 0, fe[j] = CLS_NONE;
    // a table's slot 0 holds, in w, how many slots the counter wrote; the rest are empty
    auto load_table = [&](const uint4 *t, uint32_t *k, uint32_t *cnt, uint32_t *ex) {
        const uint4 e0 = t[0];
        const uint32_t n = e0.w;
        k[0] = e0.x, cnt[0] = e0.y, ex[0] = e0.z;
#pragma unroll
        for (int j = 1; j < SU; ++j) {
            k[j] = CLS_EMPTY, cnt[j] = 0, ex[j] = CLS_NONE;
            if ((uint32_t)j < n) {
                const uint4 e = t[j];
                k[j] = e.x, cnt[j] = e.y, ex[j] = e.z;
            }
        }
    };
    // f := f followed by g: each class of f goes on through g's row for f's exit; a
    // key without its own row behaves as class "none"
    auto compose = [&](const uint32_t *gk, const uint32_t *gc, const uint32_t *ge) {
#pragma unroll
        for (int j = 0; j < SU; ++j) {
            if (fk[j] == CLS_EMPTY) continue;
            bool hit = false, hitn = false;
            uint32_t nc = 0, ne = CLS_NONE, ncn = 0, nen = CLS_NONE;
#pragma unroll
            for (int i = 0; i < SU; ++i) {
                if (!hit && gk[i] == fe[j]) hit = true, nc = gc[i], ne = ge[i];
                if (!hitn && gk[i] == CLS_NONE) hitn = true, ncn = gc[i], nen = ge[i];
            }
            if (!hit && !hitn) bad = true;
            fc[j] += hit ? nc : ncn;
            fe[j] = hit ? ne : nen;
        }
    };
    if (!ident) {
        load_table(tables + ((uint64_t)a * m + ci) * SMX, fk, fc, fe);
        for (uint32_t q = a + 1; q < b; ++q) {
            uint32_t gk[SU], gc[SU], ge[SU];
            load_table(tables + ((uint64_t)q * m + ci) * SMX, gk, gc, ge);
            compose(gk, gc, ge);
        }
    }
#pragma unroll
    for (uint32_t d = 1; d < 32; d <<= 1) {
        if (d >= G) break;  // the same on every lane
        uint32_t pk[SU], pc[SU], pe[SU];
#pragma unroll
        for (int i = 0; i < SU; ++i) {
            pk[i] = __shfl_down_sync(0xffffffffu, fk[i], d, G);
            pc[i] = __shfl_down_sync(0xffffffffu, fc[i], d, G);
            pe[i] = __shfl_down_sync(0xffffffffu, fe[i], d, G);
        }
        const bool pident = __shfl_down_sync(0xffffffffu, (int)ident, d, G) != 0;
        if ((gl & (2 * d - 1)) == 0 && gl + d < G && !pident) {
            if (ident) {
#pragma unroll
                for (int i = 0; i < SU; ++i) fk[i] = pk[i], fc[i] = pc[i], fe[i] = pe[i];
                ident = false;
            } else {
                compose(pk, pc, pe);
            }
        }
    }
    // a composition step of any lane of the group that found no row makes it fail
    const uint32_t gmask = G >= 32 ? 0xFFFFFFFFu : ((1u << G) - 1u) << (lane & ~(G - 1));
    bad = (__ballot_sync(0xffffffffu, bad) & gmask) != 0;
    if (gl == 0 && live) {
        bool found = false;
        uint32_t total = 0;
#pragma unroll
        for (int j = 0; j < SU; ++j)
            if (!found && fk[j] == CLS_NONE) found = true, total = fc[j];
        if (bad || !found) {
            redo[ci] = 1;
            atomicOr(err, ERR_TABLE);
        } else {
            out[ci] = total;
        }
    }
}

// G lanes per episode (a power of two up to 32, G = 32 / 2^k episodes per warp).  Lane
// gl of a group composes the transfer tables of its contiguous run of segments (for
// every entry class of the run's first segment); the G partial functions are then
// composed pairwise in log2(G) shuffle rounds, the tree of Concatenate steps; lane 0 of
// the group evaluates the result at class "none".  Most tables hold one or two
// classes: the warp first reads how many slots its tables use and composes over that
// many only (1, 2, 4, 8 or all), a choice the same on every lane, so the composition
// stays unrolled and free of branches.
template <int SMX>
__device__ void stitch_one(const uint4 *__restrict__ tables, uint32_t m, uint32_t P, uint32_t ci,
                           uint32_t G, bool live, uint32_t *__restrict__ out,
                           uint8_t *__restrict__ redo, uint32_t *err) {
    const uint32_t gl = threadIdx.x & (G - 1), lg = __ffs(G) - 1;
    live = live && !redo[ci];  // a flagged episode is recounted by the host
    const uint32_t a = (uint32_t)(((uint64_t)P * gl) >> lg);
    const uint32_t b = (uint32_t)(((uint64_t)P * (gl + 1)) >> lg);
    uint32_t n = 1;
    if (live)
        for (uint32_t q = a; q < b; ++q) n = max(n, tables[((uint64_t)q * m + ci) * SMX].w);
    n = __reduce_max_sync(0xffffffffu, n);
    if (n <= 1)
        stitch_run<SMX, 1>(tables, m, a, b, ci, G, gl, live, out, redo, err);
    else if (n <= 2)
        stitch_run<SMX, 2>(tables, m, a, b, ci, G, gl, live, out, redo, err);
    else if (n <= 4)
        stitch_run<SMX, (SMX < 4 ? SMX : 4)>(tables, m, a, b, ci, G, gl, live, out, redo, err);
    else if (SMX > 8 && n <= 8)
        stitch_run<SMX, (SMX < 8 ? SMX : 8)>(tables, m, a, b, ci, G, gl, live, out, redo, err);
    else
        stitch_run<SMX, SMX>(tables, m, a, b, ci, G, gl, live, out, redo, err);
}

template <int SMX>
__global__ void __launch_bounds__(256) k_stitch(const uint4 *__restrict__ tables, uint32_t m,
                                                uint32_t P, uint32_t G, uint32_t *__restrict__ out,
                                                uint8_t *__restrict__ redo, uint32_t *err) {
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, lg = __ffs(G) - 1;
    if (((gt & ~31u) >> lg) >= m) return;  // the whole warp is past the end
    const uint32_t ci = gt >> lg;
    stitch_one<SMX>(tables, m, P, ci, G, ci < m, out, redo, err);
}

// One warp per episode slot of a batch of jobs (each job its own tables and outputs).
__global__ void __launch_bounds__(256) k_stitch_batch(const CountParams *__restrict__ jobs,
                                                      const uint32_t *__restrict__ job_base,
                                                      uint32_t n_jobs, uint32_t slots,
                                                      uint32_t *err) {
    const uint32_t e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e >= slots) return;
    uint32_t lo = 0, hi = n_jobs;  // last j with job_base[j] <= e
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (job_base[mid] <= e) lo = mid;
        else hi = mid;
    }
    const CountParams &p = jobs[lo];
    const uint32_t ci = e - job_base[lo];
    stitch_one<S_MAX>(p.tables, p.m, p.P, ci, 32u, ci < p.m && p.P > 0, p.out, p.redo, err);
}

cudaError_t launch_stitch_batch(const CountParams *jobs, const uint32_t *job_base,
                                uint32_t n_jobs, uint32_t slots, uint32_t *err, cudaStream_t st) {
    if (slots == 0 || n_jobs == 0) return cudaSuccess;
    const uint32_t blocks = (uint32_t)(((uint64_t)slots * 32 + 255) / 256);
    k_stitch_batch<<<blocks, 256, 0, st>>>(jobs, job_base, n_jobs, slots, err);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_stitch(const uint4 *tables, uint32_t m, uint32_t P, uint32_t *out,
                          uint8_t *redo, uint32_t *err, cudaStream_t st, uint32_t classes) {
    if (m == 0) return cudaSuccess;
    // lanes per episode: about four segments per lane, so that a short cut (the relaxed
    // passes' 20-odd segments) takes a quarter of a warp rather than a whole one
    uint32_t G = 1;
    while (G < 32 && G * 4 < P) G <<= 1;
    const uint32_t blocks = (uint32_t)(((uint64_t)m * G + 255) / 256);
    if (classes == S_RECOUNT)
        k_stitch<S_RECOUNT><<<blocks, 256, 0, st>>>(tables, m, P, G, out, redo, err);
    else if (classes == S_MAX)
        k_stitch<S_MAX><<<blocks, 256, 0, st>>>(tables, m, P, G, out, redo, err);
    else
        return cudaErrorInvalidValue;
    note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ candidate validation
// info[0] |= 1 << len for every candidate; info[1] += candidates with a repeated type.
__global__ void k_validate_cands(const fem_episode *__restrict__ c, const uint32_t *gather,
                                 uint32_t m, uint32_t K, uint32_t n_ivl, uint32_t *info,
                                 uint32_t *err) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t lenbit = 0, rep = 0, bad = 0, brk = 0;
    if (i < m) {
        const fem_episode e = ld_ep(c, gather ? gather[i] : i);
        const uint32_t N = e.len;
        // a run of candidates sharing the prefix that a last node extends ends here
        if (i > 0) {
            const fem_episode q = ld_ep(c, gather ? gather[i - 1] : i - 1);
            brk = q.len != N;
            for (uint32_t k = 0; k + 1 < N && k < FEM_MAX_LEN; ++k) brk |= q.types[k] != e.types[k];
            for (uint32_t k = 0; k + 2 < N && k < FEM_MAX_LEN - 1; ++k) brk |= q.ivl[k] != e.ivl[k];
        }
        if (N < 1 || N > FEM_MAX_LEN) {
            bad = ERR_BADEP;
        } else {
            lenbit = 1u << N;
            for (uint32_t k = 0; k < N; ++k)
                if (e.types[k] >= K) bad = ERR_BADEP;
            for (uint32_t k = 0; k + 1 < N; ++k)
                if (e.ivl[k] >= n_ivl) bad = ERR_BADEP;
            for (uint32_t a = 0; a < N; ++a)
                for (uint32_t b2 = a + 1; b2 < N; ++b2)
                    if (e.types[a] == e.types[b2]) rep = 1;
        }
    }
    lenbit = __reduce_or_sync(0xffffffffu, lenbit);
    rep = __reduce_add_sync(0xffffffffu, rep);
    bad = __reduce_or_sync(0xffffffffu, bad);
    brk = __reduce_add_sync(0xffffffffu, brk);
    if ((threadIdx.x & 31) == 0) {
        if (lenbit) atomicOr(&info[0], lenbit);
        if (rep) atomicAdd(&info[1], rep);
        if (brk) atomicAdd(&info[2], brk);
        if (bad) atomicOr(err, bad);
    }
}

cudaError_t launch_validate_cands(const fem_episode *c, const uint32_t *gather, uint32_t m,
                                  uint32_t K, uint32_t n_ivl, uint32_t *info, uint32_t *err,
                                  cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_validate_cands<<<(m + 255) / 256, 256, 0, st>>>(c, gather, m, K, n_ivl, info, err);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_len_flags(const fem_episode *__restrict__ c, const uint32_t *gather,
                            uint32_t m, uint32_t N, uint8_t *__restrict__ flags) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) flags[i] = ld_ep(c, gather ? gather[i] : i).len == N;
}

// flags[i] = 1 if candidate i (gathered) has a repeated type, xor `invert`
__global__ void k_repeat_flags(const fem_episode *__restrict__ c, const uint32_t *__restrict__ gather,
                               uint32_t m, uint32_t invert, uint8_t *__restrict__ flags) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const fem_episode e = c[gather ? gather[i] : i];
    uint32_t rep = 0;
    for (uint32_t a = 0; a < e.len && a < FEM_MAX_LEN; ++a)
        for (uint32_t b = a + 1; b < e.len && b < FEM_MAX_LEN; ++b) rep |= e.types[a] == e.types[b];
    flags[i] = (uint8_t)(rep ^ invert);
}

cudaError_t launch_repeat_flags(const fem_episode *c, const uint32_t *gather, uint32_t m, bool invert,
                                uint8_t *flags, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_repeat_flags<<<(m + 255) / 256, 256, 0, st>>>(c, gather, m, invert ? 1u : 0u, flags);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_len_flags(const fem_episode *c, const uint32_t *gather, uint32_t m, uint32_t N,
                             uint8_t *flags, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_len_flags<<<(m + 255) / 256, 256, 0, st>>>(c, gather, m, N, flags);
    note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ stable compaction
size_t compact_scratch_words(uint32_t m) { return compact_scratch_words_for(m); }

// (one thread) the count and the error word into the mapped host words, if any
__device__ __forceinline__ void publish(const Publish &pub, uint32_t count) {
    if (!pub.host) return;
    volatile uint32_t *h = pub.host;
    h[0] = count;
    h[1] = *reinterpret_cast<const volatile uint32_t *>(pub.err);
    __threadfence_system();
    h[2] = pub.seq;
}

__global__ void k_set_count(uint32_t *count, Publish pub) {
    *count = 0;
    publish(pub, 0);
}

__global__ void __launch_bounds__(CT) k_keep_count(const uint32_t *vals, const uint8_t *flags,
                                                    uint32_t theta, uint32_t m,
                                                    uint32_t *blocksum) {
    const uint32_t base = blockIdx.x * CB + threadIdx.x * CI;
    uint32_t c = 0;
#pragma unroll
    for (uint32_t k = 0; k < CI; ++k)
        if (base + k < m) c += keep_at(vals, flags, theta, base + k);
    uint32_t tot;
    block_exclusive_scan(c, &tot);
    if (threadIdx.x == 0) blocksum[blockIdx.x] = tot;
}

// In-place exclusive scan of a[0..nb) by one block of 1024 threads; *total = sum.
__global__ void __launch_bounds__(1024) k_scan_small(uint32_t *a, uint32_t nb, uint32_t *total,
                                                     Publish pub) {
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? a[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, &tot);
        if (i < nb) a[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
    if (threadIdx.x == 0) publish(pub, carry);
}

__global__ void __launch_bounds__(CT) k_keep_scatter(const uint32_t *vals, const uint8_t *flags,
                                                      uint32_t theta, uint32_t m,
                                                      const uint32_t *blockoff, uint32_t *idx) {
    const uint32_t base = blockIdx.x * CB + threadIdx.x * CI;
    bool kp[CI];
    uint32_t c = 0;
#pragma unroll
    for (uint32_t k = 0; k < CI; ++k) {
        kp[k] = base + k < m && keep_at(vals, flags, theta, base + k);
        c += kp[k];
    }
    uint32_t pos = blockoff[blockIdx.x] + block_exclusive_scan(c, nullptr);
#pragma unroll
    for (uint32_t k = 0; k < CI; ++k)
        if (kp[k]) idx[pos++] = base + k;
}

// Up to ST * SI items (the candidate sets of most levels) are compacted or scanned
// by one block of ST threads, each on a contiguous run of SI items: one launch
// instead of three, which matters in the stretches between host waits, where the
// host issues short kernels one after another.
constexpr uint32_t ST = 1024, SI = 16;
static_assert(SI == 16, "k_compact_small takes half a keep-bit word per thread");

__global__ void __launch_bounds__(ST) k_compact_small(const uint32_t *vals, const uint8_t *flags,
                                                      uint32_t theta, uint32_t m, uint32_t *idx,
                                                      uint32_t *count, Publish pub) {
    // keep bits, one word per 32 items, from coalesced reads (item r * ST + thread)
    __shared__ uint32_t keep_bits[ST * SI / 32];
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (uint32_t r = 0; r < SI; ++r) {
        const uint32_t i = r * ST + threadIdx.x;
        const uint32_t w = __ballot_sync(0xffffffffu, i < m && keep_at(vals, flags, theta, i));
        if (lane == 0) keep_bits[i >> 5] = w;
    }
    __syncthreads();
    // thread t then owns items t * SI .. t * SI + SI - 1 (SI = 16: half a word)
    const uint32_t base = threadIdx.x * SI;
    uint32_t bits = (keep_bits[base >> 5] >> (base & 31u)) & 0xFFFFu;
    uint32_t tot;
    uint32_t pos = block_exclusive_scan(__popc(bits), &tot);
    while (bits) {
        const uint32_t k = __ffs(bits) - 1;
        bits &= bits - 1;
        idx[pos++] = base + k;
    }
    if (threadIdx.x == 0) {
        *count = tot;
        publish(pub, tot);
    }
}

__global__ void __launch_bounds__(ST) k_scan_one_block(const uint32_t *in, uint32_t m,
                                                       uint32_t *out, uint32_t *total,
                                                       Publish pub) {
    const uint32_t base = threadIdx.x * SI;
    uint32_t v[SI], c = 0;
#pragma unroll
    for (uint32_t k = 0; k < SI; ++k) {
        v[k] = base + k < m ? in[base + k] : 0u;
        c += v[k];
    }
    uint32_t tot;
    uint32_t pos = block_exclusive_scan(c, &tot);
#pragma unroll
    for (uint32_t k = 0; k < SI; ++k) {
        if (base + k < m) out[base + k] = pos;
        pos += v[k];
    }
    if (threadIdx.x == 0 && total) *total = tot;
    if (threadIdx.x == 0) publish(pub, tot);
}

cudaError_t launch_compact(const uint32_t *vals, const uint8_t *flags, uint32_t theta, uint32_t m,
                           uint32_t *idx_out, uint32_t *count_out, uint32_t *scratch,
                           cudaStream_t st, Publish pub) {
    if (m == 0) {
        if (!pub.host) return cudaMemsetAsync(count_out, 0, sizeof(uint32_t), st);
        k_set_count<<<1, 1, 0, st>>>(count_out, pub);
        note_launch();
        return cudaGetLastError();
    }
    if (m <= ST * SI) {
        k_compact_small<<<1, ST, 0, st>>>(vals, flags, theta, m, idx_out, count_out, pub);
        note_launch();
        return cudaGetLastError();
    }
    const uint32_t nb = (m + CB - 1) / CB;
    k_keep_count<<<nb, CT, 0, st>>>(vals, flags, theta, m, scratch);
    note_launch();
    k_scan_small<<<1, 1024, 0, st>>>(scratch, nb, count_out, pub);
    note_launch();
    k_keep_scatter<<<nb, CT, 0, st>>>(vals, flags, theta, m, scratch, idx_out);
    note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ exclusive scan of counts
__global__ void __launch_bounds__(CT) k_sum_blocks(const uint32_t *in, uint32_t m,
                                                    uint32_t *blocksum) {
    const uint32_t base = blockIdx.x * CB + threadIdx.x * CI;
    uint32_t c = 0;
#pragma unroll
    for (uint32_t k = 0; k < CI; ++k)
        if (base + k < m) c += in[base + k];
    uint32_t tot;
    block_exclusive_scan(c, &tot);
    if (threadIdx.x == 0) blocksum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(CT) k_scan_apply(const uint32_t *in, uint32_t m,
                                                    const uint32_t *blockoff, uint32_t *out) {
    const uint32_t base = blockIdx.x * CB + threadIdx.x * CI;
    uint32_t v[CI], c = 0;
#pragma unroll
    for (uint32_t k = 0; k < CI; ++k) {
        v[k] = base + k < m ? in[base + k] : 0u;
        c += v[k];
    }
    uint32_t pos = blockoff[blockIdx.x] + block_exclusive_scan(c, nullptr);
#pragma unroll
    for (uint32_t k = 0; k < CI; ++k) {
        if (base + k < m) out[base + k] = pos;
        pos += v[k];
    }
}

cudaError_t launch_exclusive_scan(const uint32_t *in, uint32_t m, uint32_t *out, uint32_t *total,
                                  uint32_t *scratch, cudaStream_t st, Publish pub) {
    if (m == 0) {
        if (!pub.host) return cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        k_set_count<<<1, 1, 0, st>>>(total, pub);
        note_launch();
        return cudaGetLastError();
    }
    if (m <= ST * SI) {
        k_scan_one_block<<<1, ST, 0, st>>>(in, m, out, total, pub);
        note_launch();
        return cudaGetLastError();
    }
    const uint32_t nb = (m + CB - 1) / CB;
    k_sum_blocks<<<nb, CT, 0, st>>>(in, m, scratch);
    note_launch();
    k_scan_small<<<1, 1024, 0, st>>>(scratch, nb, total, pub);
    note_launch();
    k_scan_apply<<<nb, CT, 0, st>>>(in, m, scratch, out);
    note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ gathers and scatters
__global__ void k_gather_ep(const fem_episode *__restrict__ src, const uint32_t *__restrict__ idx,
                            uint32_t m, fem_episode *__restrict__ dst,
                            const uint32_t *__restrict__ vals, uint32_t *__restrict__ vdst) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint32_t j = idx[i];
    if (dst) st_ep(dst, i, ld_ep(src, j));
    if (vdst) vdst[i] = vals[j];
}

cudaError_t launch_gather_episodes(const fem_episode *src, const uint32_t *idx, uint32_t m,
                                   fem_episode *dst, const uint32_t *vals, uint32_t *vals_dst,
                                   cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_gather_ep<<<(m + 255) / 256, 256, 0, st>>>(src, idx, m, dst, vals, vals_dst);
    note_launch();
    return cudaGetLastError();
}

// The frequent set of a level in one launch: F[i] = cands[surv[idx[i]]] and
// fcnt[i] = counts[idx[i]], where surv lists the survivors of the first pass and idx
// the survivors of the second (both ascending, so F keeps the candidates' order).
__global__ void k_gather_frequent(const fem_episode *__restrict__ cands,
                                  const uint32_t *__restrict__ surv, const uint32_t *__restrict__ idx,
                                  uint32_t f, const uint32_t *__restrict__ counts,
                                  fem_episode *__restrict__ F, uint32_t *__restrict__ fcnt) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= f) return;
    const uint32_t j = idx[i];
    st_ep(F, i, ld_ep(cands, surv[j]));
    fcnt[i] = counts[j];
}

cudaError_t launch_gather_frequent(const fem_episode *cands, const uint32_t *surv,
                                   const uint32_t *idx, uint32_t f, const uint32_t *counts,
                                   fem_episode *F, uint32_t *fcnt, cudaStream_t st) {
    if (f == 0) return cudaSuccess;
    k_gather_frequent<<<(f + 255) / 256, 256, 0, st>>>(cands, surv, idx, f, counts, F, fcnt);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_scatter_u32(const uint32_t *__restrict__ src, const uint32_t *__restrict__ idx,
                              uint32_t m, uint32_t *__restrict__ dst) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) dst[idx[i]] = src[i];
}

cudaError_t launch_scatter_u32(const uint32_t *src, const uint32_t *idx, uint32_t m,
                               uint32_t *dst, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_scatter_u32<<<(m + 255) / 256, 256, 0, st>>>(src, idx, m, dst);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_scatter_dev(const uint32_t *__restrict__ src, const uint32_t *__restrict__ idx,
                              const uint32_t *__restrict__ m_dev, uint32_t m_max,
                              uint32_t *__restrict__ dst, uint8_t *__restrict__ flags) {
    const uint32_t m = min(*m_dev, m_max);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        dst[idx[i]] = src[i];
        if (flags) flags[idx[i]] = 1;
    }
}

cudaError_t launch_scatter_dev(const uint32_t *src, const uint32_t *idx, const uint32_t *m_dev,
                               uint32_t m_max, uint32_t *dst, uint8_t *flags, cudaStream_t st) {
    if (m_max == 0) return cudaSuccess;
    const uint32_t blocks = (m_max + 255) / 256 < 2048 ? (m_max + 255) / 256 : 2048;
    k_scatter_dev<<<blocks, 256, 0, st>>>(src, idx, m_dev, m_max, dst, flags);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_fill_flags(const uint32_t *__restrict__ idx, uint32_t m,
                             uint8_t *__restrict__ flags) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) flags[idx[i]] = 1;
}

cudaError_t launch_fill_flags(const uint32_t *idx, uint32_t m, uint8_t *flags, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_fill_flags<<<(m + 255) / 256, 256, 0, st>>>(idx, m, flags);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_compose_idx(const uint32_t *__restrict__ outer, const uint32_t *__restrict__ inner,
                              uint32_t m, uint32_t *__restrict__ dst) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) dst[i] = outer ? outer[inner[i]] : inner[i];
}

cudaError_t launch_compose_idx(const uint32_t *outer, const uint32_t *inner, uint32_t m,
                               uint32_t *dst, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_compose_idx<<<(m + 255) / 256, 256, 0, st>>>(outer, inner, m, dst);
    note_launch();
    return cudaGetLastError();
}

// Work measure of a counting pass: sum over the (gathered) candidates of the events
// of their types, from the type histogram; one 64-bit atomic per warp.
__global__ void k_touched(const fem_episode *__restrict__ cands, const uint32_t *__restrict__ gather,
                          uint32_t m, const uint32_t *__restrict__ hist,
                          unsigned long long *out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < m) {
        const fem_episode e = cands[gather ? gather[i] : i];
        for (uint32_t k = 0; k < e.len && k < FEM_MAX_LEN; ++k) v += hist[e.types[k]];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31u) == 0 && v) atomicAdd(out, v);
}

cudaError_t launch_touched(const fem_episode *cands, const uint32_t *gather, uint32_t m,
                           const uint32_t *hist, unsigned long long *out, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_touched<<<(m + 255) / 256, 256, 0, st>>>(cands, gather, m, hist, out);
    note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ level-wise generation
// Frequent types: hist[a] >= theta, in increasing type order (one block, K <= 256).
__global__ void k_type_filter(const uint32_t *hist, uint32_t K, uint32_t theta, uint32_t *ftypes,
                              uint32_t *fcount) {
    const uint32_t a = threadIdx.x;
    const uint32_t keep = a < K && hist[a] >= theta;
    uint32_t tot;
    const uint32_t pos = block_exclusive_scan(keep, &tot);
    if (keep) ftypes[pos] = a;
    if (threadIdx.x == 0) *fcount = tot;
}

cudaError_t launch_type_filter(const uint32_t *hist, uint32_t K, uint32_t theta, uint32_t *ftypes,
                               uint32_t *fcount, cudaStream_t st) {
    k_type_filter<<<1, 256, 0, st>>>(hist, K, theta, ftypes, fcount);
    note_launch();
    return cudaGetLastError();
}

// Level 2: ordered pairs (a, b) of frequent types, a != b unless `repeats`, once per
// interval, in canonical order (a, interval, b).
__global__ void k_level2(const uint32_t *__restrict__ ftypes, uint32_t f, uint32_t n_ivl,
                         uint32_t repeats, fem_episode *__restrict__ out) {
    const uint32_t nb = repeats ? f : f - 1;  // second types per first type
    const uint64_t m = (uint64_t)f * n_ivl * nb;
    const uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (c >= m) return;
    const uint64_t per_a = (uint64_t)n_ivl * nb;
    const uint32_t ai = (uint32_t)(c / per_a);
    const uint32_t r = (uint32_t)(c % per_a);
    const uint32_t iv = r / nb;
    const uint32_t bj = r % nb;
    const uint32_t bi = (repeats || bj < ai) ? bj : bj + 1;
    fem_episode e;
    memset(&e, 0, sizeof(e));
    e.types[0] = (uint8_t)ftypes[ai];
    e.types[1] = (uint8_t)ftypes[bi];
    e.ivl[0] = (uint8_t)iv;
    e.len = 2;
    st_ep(out, c, e);
}

cudaError_t launch_level2(const uint32_t *ftypes, uint32_t f, uint32_t n_ivl, bool repeats,
                          fem_episode *out, cudaStream_t st) {
    if (f < (repeats ? 1u : 2u) || n_ivl == 0) return cudaSuccess;
    const uint64_t m = (uint64_t)f * n_ivl * (repeats ? f : f - 1);
    k_level2<<<(uint32_t)((m + 255) / 256), 256, 0, st>>>(ftypes, f, n_ivl, repeats ? 1u : 0u,
                                                          out);
    note_launch();
    return cudaGetLastError();
}

namespace {
// Compare beta's first N-1 nodes (with its first N-2 intervals) against alpha's
// last N-1 nodes (with its last N-2 intervals), in interleaved order.
__device__ __forceinline__ int cmp_prefix_suffix(const fem_episode &b, const fem_episode &a,
                                                 uint32_t N) {
    for (uint32_t k = 0; k + 1 < N; ++k) {
        int d = (int)b.types[k] - (int)a.types[k + 1];
        if (d) return d;
        if (k + 2 < N) {
            d = (int)b.ivl[k] - (int)a.ivl[k + 1];
            if (d) return d;
        }
    }
    return 0;
}
// [lo, hi) of the frequent episodes whose prefix equals alpha's suffix.
__device__ void join_range(const fem_episode *F, uint32_t f, uint32_t N, const fem_episode &a,
                           uint32_t *lo_out, uint32_t *hi_out) {
    uint32_t lo = 0, hi = f;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (cmp_prefix_suffix(ld_ep(F, mid), a, N) < 0) lo = mid + 1;
        else hi = mid;
    }
    uint32_t lo2 = lo, hi2 = f;
    while (lo2 < hi2) {
        const uint32_t mid = (lo2 + hi2) >> 1;
        if (cmp_prefix_suffix(ld_ep(F, mid), a, N) <= 0) lo2 = mid + 1;
        else hi2 = mid;
    }
    *lo_out = lo;
    *hi_out = lo2;
}
__device__ __forceinline__ bool has_type(const fem_episode &a, uint32_t N, uint32_t x) {
    bool h = false;
    for (uint32_t k = 0; k < N; ++k) h |= a.types[k] == x;
    return h;
}
}  // namespace

// Join (level N -> N+1): alpha joins beta when alpha minus its first node equals
// beta minus its last node; the child appends beta's last edge and node, whose
// type must be new to alpha.  F is in canonical order, so the betas of one
// alpha are contiguous and the children come out in canonical order.
// Up to this many frequent episodes (48 KB) are staged in each block's shared memory,
// so the binary searches and the scans of matching ranges read no global memory.
constexpr uint32_t JOIN_SMEM_MAX = 3072;
// One warp per alpha: its lanes take the matching betas 32 at a time, so an alpha
// with a long range (a type that starts many frequent episodes) does not hold up the
// launch (level 2 -> 3 of the 64-type recording: 66 us with one thread per alpha).
constexpr uint32_t JOIN_WARPS = 8;  // warps per block

__device__ __forceinline__ const fem_episode *stage_frequent(const fem_episode *F, uint32_t f) {
    extern __shared__ uint4 s_freq[];
    if (f > JOIN_SMEM_MAX) return F;  // uniform over the launch
    for (uint32_t j = threadIdx.x; j < f; j += blockDim.x)
        s_freq[j] = reinterpret_cast<const uint4 *>(F)[j];
    __syncthreads();
    return reinterpret_cast<const fem_episode *>(s_freq);
}

// The child alpha + beta's last node is kept if that type is new to alpha, or
// always when `repeats`.
__global__ void __launch_bounds__(JOIN_WARPS * 32)
    k_join_count(const fem_episode *__restrict__ Fg, uint32_t f, uint32_t N, uint32_t repeats,
                 uint32_t *__restrict__ cnt) {
    const fem_episode *F = stage_frequent(Fg, f);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nw = gridDim.x * JOIN_WARPS;
    for (uint32_t i = blockIdx.x * JOIN_WARPS + (threadIdx.x >> 5); i < f; i += nw) {
        const fem_episode a = ld_ep(F, i);
        uint32_t lo, hi;
        join_range(F, f, N, a, &lo, &hi);  // the same on every lane
        uint32_t c = 0;
        for (uint32_t j = lo + lane; j < hi; j += 32)
            c += repeats || !has_type(a, N, ld_ep(F, j).types[N - 1]);
        c = __reduce_add_sync(0xFFFFFFFFu, c);
        if (lane == 0) cnt[i] = c;
    }
}

__global__ void __launch_bounds__(JOIN_WARPS * 32)
    k_join_emit(const fem_episode *__restrict__ Fg, uint32_t f, uint32_t N, uint32_t repeats,
                const uint32_t *__restrict__ off, fem_episode *__restrict__ out) {
    const fem_episode *F = stage_frequent(Fg, f);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t nw = gridDim.x * JOIN_WARPS;
    for (uint32_t i = blockIdx.x * JOIN_WARPS + (threadIdx.x >> 5); i < f; i += nw) {
        const fem_episode a = ld_ep(F, i);
        uint32_t lo, hi;
        join_range(F, f, N, a, &lo, &hi);
        uint32_t pos = off[i];
        for (uint32_t j0 = lo; j0 < hi; j0 += 32) {  // warp-uniform trip count
            const uint32_t j = j0 + lane;
            bool keep = false;
            fem_episode b;
            if (j < hi) {
                b = ld_ep(F, j);
                keep = repeats || !has_type(a, N, b.types[N - 1]);
            }
            // kept children of this batch go out in beta order, one per lane
            const uint32_t kept = __ballot_sync(0xFFFFFFFFu, keep);
            if (keep) {
                fem_episode c = a;
                c.types[N] = b.types[N - 1];
                c.ivl[N - 1] = b.ivl[N - 2];
                c.len = (uint8_t)(N + 1);
                st_ep(out, pos + __popc(kept & below), c);
            }
            pos += __popc(kept);
        }
    }
}

namespace {
// Blocks of a join launch: one warp per alpha, at most `per_sm` blocks per SM (with F
// staged, every block copies it once; without, more blocks hide global latency).
uint32_t join_blocks(uint32_t f, int sm_count) {
    const uint32_t per_sm = f <= JOIN_SMEM_MAX ? 1u : 8u;
    const uint32_t cap = (uint32_t)std::max(sm_count, 1) * per_sm;
    return std::max(1u, std::min((f + JOIN_WARPS - 1) / JOIN_WARPS, cap));
}
}  // namespace

cudaError_t launch_join_count(const fem_episode *F, uint32_t f, uint32_t N, bool repeats,
                              uint32_t *cnt, int sm_count, cudaStream_t st) {
    if (f == 0) return cudaSuccess;
    const size_t sm = f <= JOIN_SMEM_MAX ? (size_t)f * sizeof(fem_episode) : 0;
    k_join_count<<<join_blocks(f, sm_count), JOIN_WARPS * 32, sm, st>>>(F, f, N, repeats ? 1u : 0u,
                                                                         cnt);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_join_emit(const fem_episode *F, uint32_t f, uint32_t N, bool repeats,
                             const uint32_t *off, fem_episode *out, int sm_count, cudaStream_t st) {
    if (f == 0) return cudaSuccess;
    const size_t sm = f <= JOIN_SMEM_MAX ? (size_t)f * sizeof(fem_episode) : 0;
    k_join_emit<<<join_blocks(f, sm_count), JOIN_WARPS * 32, sm, st>>>(
        F, f, N, repeats ? 1u : 0u, off, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fem
