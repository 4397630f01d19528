// fem_stream.cu -- staging of a resident event stream (load_stream).
//
// Validates the stream of Def. 2.1 (times non-decreasing, types < K) and builds
// the chunked per-type layout every counting kernel reads: for each chunk of
// CHUNK consecutive events, the events stably grouped by type with their time
// and local index, plus the group offsets.  Within a group the events keep
// stream order, so a thread that merges its episode's groups by local index
// sees exactly the subsequence of the stream made of its episode's types.
#include <algorithm>

#include "fem_internal.cuh"

namespace fem {

// One block of 256 threads per chunk.  Warp w ranks events [256w, 256w+256) of the
// chunk within their type (match.any per 32-event round), the per-(warp, type)
// counts are scanned type-major, and each event is written to its slot.  The events
// are read from (t, ty); with `err` the block also checks them (types < K, times
// non-decreasing, the pair across the chunk's end included) and ORs the findings in;
// with `t_out` it also copies them there (the library's own copy of a stream loaded
// from device memory), so that a load takes one kernel.  Event types are bytes, so
// the grouping stays in bounds whatever K is; a load that finds bad events fails.
__global__ void __launch_bounds__(256) k_bucket(const uint32_t *__restrict__ t,
                                                const uint8_t *__restrict__ ty, uint64_t n,
                                                uint32_t K, uint32_t offs, uint32_t n_chunks,
                                                uint2 *__restrict__ bev,
                                                uint16_t *__restrict__ boff,
                                                uint32_t *__restrict__ cfirst,
                                                uint32_t *__restrict__ hist, uint32_t c0,
                                                uint32_t *err, uint32_t *__restrict__ t_out,
                                                uint8_t *__restrict__ ty_out) {
    __shared__ uint16_t wcnt[8][256];
    __shared__ uint32_t tbase[257];
    __shared__ uint32_t wsum[8];
    const uint32_t c = c0 + blockIdx.x;
    const uint64_t base = (uint64_t)c * CHUNK;
    const uint32_t cnt = (uint32_t)min((uint64_t)CHUNK, n - base);
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (uint32_t i = threadIdx.x; i < 8 * 256; i += 256) (&wcnt[0][0])[i] = 0;
    __syncthreads();

    uint32_t myty[8], myrank[8], bad = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const uint32_t li = w * 256 + r * 32 + lane;
        const bool valid = li < cnt;
        const uint32_t v = valid ? ty[base + li] : 0u;
        const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
        myty[r] = v;
        myrank[r] = 0;
        if (valid && err) {
            const uint64_t gi = base + li;
            if (v >= K) bad |= ERR_TYPE;
            if (gi + 1 < n && t[gi] > t[gi + 1]) bad |= ERR_UNSORTED;
        }
        if (valid && t_out) {
            t_out[base + li] = t[base + li];
            ty_out[base + li] = (uint8_t)v;
        }
        if (valid) {
            const uint32_t peers = __match_any_sync(vmask, v);
            const uint32_t below = __popc(peers & ((1u << lane) - 1u));
            const uint32_t prev = wcnt[w][v];
            __syncwarp(vmask);
            if (below == 0) wcnt[w][v] = (uint16_t)(prev + __popc(peers));
            myrank[r] = prev + below;
        }
        __syncwarp();
    }
    __syncthreads();

    // per type (thread = type value): per-warp exclusive prefix and total
    const uint32_t tv = threadIdx.x;
    uint32_t tot = 0;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) {
        const uint32_t x = wcnt[ww][tv];
        wcnt[ww][tv] = (uint16_t)tot;
        tot += x;
    }
    // exclusive scan of tot over the 256 type values
    uint32_t inc = tot;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= (uint32_t)d) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t woff = 0;
    for (uint32_t ww = 0; ww < w; ++ww) woff += wsum[ww];
    tbase[tv] = woff + inc - tot;
    if (tv == 255) tbase[256] = woff + inc;
    if (hist && tv < K && tot) atomicAdd(&hist[tv], tot);
    __syncthreads();

#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const uint32_t li = w * 256 + r * 32 + lane;
        if (li < cnt) {
            const uint32_t pos = tbase[myty[r]] + wcnt[w][myty[r]] + myrank[r];
            bev[base + pos] = make_uint2(t[base + li], li);
        }
    }
    for (uint32_t k = threadIdx.x; k < offs; k += 256)
        boff[(uint64_t)c * offs + k] = (uint16_t)(k <= K ? tbase[k] : cnt);
    if (threadIdx.x == 0) {
        cfirst[c] = t[base];
        if (c + 1 == n_chunks) cfirst[n_chunks] = 0xFFFFFFFFu;
    }
    if (err) {
        bad = __reduce_or_sync(0xffffffffu, bad);
        if (bad && lane == 0) atomicOr(err, bad);
    }
}

cudaError_t launch_load_stream(StreamDev &s, cudaStream_t st, uint32_t *d_err,
                               const uint32_t *src_t, const uint8_t *src_type) {
    if (s.n == 0) return cudaSuccess;
    if (src_t)  // device input: read it where it is and copy it while grouping
        k_bucket<<<s.n_chunks, 256, 0, st>>>(src_t, src_type, s.n, s.K, s.offs, s.n_chunks, s.bev,
                                             s.boff, s.cfirst, s.hist, 0, d_err, s.t, s.type);
    else
        k_bucket<<<s.n_chunks, 256, 0, st>>>(s.t, s.type, s.n, s.K, s.offs, s.n_chunks, s.bev,
                                             s.boff, s.cfirst, s.hist, 0, d_err, nullptr, nullptr);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_bucket_chunks(StreamDev &s, uint32_t c0, uint32_t c1, cudaStream_t st,
                                 uint32_t *d_err) {
    if (c1 <= c0) return cudaSuccess;
    k_bucket<<<c1 - c0, 256, 0, st>>>(s.t, s.type, s.n, s.K, s.offs, s.n_chunks, s.bev, s.boff,
                                      s.cfirst, nullptr, c0, d_err, nullptr, nullptr);
    note_launch();
    return cudaGetLastError();
}

// hist[ty[i]] += sign for the n events (types >= K are skipped: a load that holds
// them fails and is undone)
__global__ void __launch_bounds__(256) k_hist_add(const uint8_t *__restrict__ ty, uint64_t n,
                                                  uint32_t K, int sign, uint32_t *hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (uint64_t)gridDim.x * 256)
        atomicAdd(&h[ty[i]], 1u);
    __syncthreads();
    const uint32_t v = h[threadIdx.x];
    if (v && threadIdx.x < K) atomicAdd(&hist[threadIdx.x], sign > 0 ? v : 0u - v);
}

cudaError_t launch_hist_add(const uint8_t *ty, uint64_t n, uint32_t K, int sign, uint32_t *hist,
                            cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 1024);
    k_hist_add<<<(uint32_t)blocks, 256, 0, st>>>(ty, n, K, sign, hist);
    note_launch();
    return cudaGetLastError();
}

// What a load reads back, into mapped pinned host words: the error word, the last time
// and the K type counts, then (after one system-wide fence) the sequence number the host
// watches for.  The block stages the counts in shared memory and one thread writes
// them all: the writes to host memory are posted, and a single fence is cheaper than one
// per thread (a fence waits for every earlier write of its thread to reach the host).
__global__ void __launch_bounds__(256) k_publish_load(const uint32_t *err, const uint32_t *t_last,
                                                      const uint32_t *hist, uint32_t K,
                                                      uint32_t *host, uint32_t seq_word,
                                                      uint32_t seq) {
    __shared__ uint32_t hs[256];  // K <= 256
    for (uint32_t a = threadIdx.x; a < K; a += blockDim.x) hs[a] = hist[a];
    __syncthreads();
    if (threadIdx.x != 0) return;
    volatile uint32_t *h = host;
    for (uint32_t a = 0; a < K; ++a) h[2 + a] = hs[a];
    h[0] = *reinterpret_cast<const volatile uint32_t *>(err);
    h[1] = t_last ? *t_last : 0u;
    __threadfence_system();
    h[seq_word] = seq;
}

cudaError_t launch_publish_load(const uint32_t *err, const uint32_t *t_last, const uint32_t *hist,
                                uint32_t K, uint32_t *host, uint32_t seq_word, uint32_t seq,
                                cudaStream_t st) {
    if (K > 256) return cudaErrorInvalidValue;
    k_publish_load<<<1, 256, 0, st>>>(err, t_last, hist, K, host, seq_word, seq);
    note_launch();
    return cudaGetLastError();
}

// Capacity table: cap[a * nh + j] = the most type-a events inside one closed window of
// length h[j].  A fullest window can start at one of its events, so one thread per
// (chunk, type) takes the events of its group in turn and, for each width, walks a
// second pointer forward through the type's groups of this and the following chunks
// while the times stay within h of the current event (two pointers: the forward one
// never moves back within the thread's group); the per-thread maxima meet by atomicMax.
// With `dense`, dense[a * nh + j] also counts the type-a events whose window of length
// h[j] holds more than `over` events (how often a bound is approached, not only whether).
__global__ void __launch_bounds__(256) k_capacity(const uint2 *__restrict__ bev,
                                                  const uint16_t *__restrict__ boff, uint32_t offs,
                                                  uint32_t n_chunks, uint32_t K,
                                                  const uint32_t *__restrict__ h, uint32_t nh,
                                                  uint32_t *__restrict__ cap, uint32_t over,
                                                  uint32_t *__restrict__ dense) {
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (uint64_t)n_chunks * K) return;
    const uint32_t c = (uint32_t)(gid / K), a = (uint32_t)(gid % K);
    const uint32_t g0 = boff[(uint64_t)c * offs + a], g1 = boff[(uint64_t)c * offs + a + 1];
    if (g0 == g1) return;
    const uint2 *ev = bev + (uint64_t)c * CHUNK;
    for (uint32_t j = 0; j < nh; ++j) {
        const uint64_t w = h[j];
        // forward pointer: chunk fc, index fk in that chunk's type-a group [fk, f1)
        uint32_t fc = c, fk = g0, f1 = g1;
        uint32_t ahead = 0, best = 0, n_over = 0;  // events in [current, forward pointer)
        for (uint32_t k = g0; k < g1; ++k) {
            const uint64_t lim = (uint64_t)ev[k].x + w;
            for (;;) {
                while (fk == f1 && fc + 1 < n_chunks) {  // next chunk's group of type a
                    ++fc;
                    fk = boff[(uint64_t)fc * offs + a];
                    f1 = boff[(uint64_t)fc * offs + a + 1];
                }
                if (fk == f1 || bev[(uint64_t)fc * CHUNK + fk].x > lim) break;
                ++fk;
                ++ahead;
            }
            best = max(best, ahead);
            n_over += ahead > over;
            --ahead;  // the current event leaves the window's start
        }
        atomicMax(&cap[a * nh + j], best);
        if (dense && n_over) atomicAdd(&dense[a * nh + j], n_over);
    }
}

cudaError_t launch_capacity(const StreamDev &s, const uint32_t *h, uint32_t nh, uint32_t *cap,
                            cudaStream_t st, uint32_t over, uint32_t *dense) {
    const uint64_t threads = (uint64_t)s.n_chunks * s.K;
    if (threads == 0 || nh == 0) return cudaSuccess;
    k_capacity<<<(uint32_t)((threads + 255) / 256), 256, 0, st>>>(s.bev, s.boff, s.offs,
                                                                   s.n_chunks, s.K, h, nh, cap,
                                                                   over, dense);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fem
