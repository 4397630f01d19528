// fem_internal.cuh -- internal declarations shared by the libfem.so translation units.
//
// Device layout of a resident event stream (built by fem_load_stream):
//   t[n], type[n]             the stream as given (Def. 2.1), SoA
//   bev[n_chunks * CHUNK]     per chunk of CHUNK consecutive events, the events
//                             stably grouped by type: (t, local index in chunk)
//   boff[n_chunks * offs]     per chunk, the start of each type's group (uint16),
//                             boff[c*offs + K] = events in the chunk; padded to a
//                             16-byte multiple so one bulk copy moves a chunk's table
//   cfirst[n_chunks + 1]      time of the first event of each chunk (+ UINT32_MAX)
//   hist[K]                   events per type (the level-1 counts)
// A counting block stages one chunk at a time into shared memory with a bulk
// (TMA) copy; each thread then walks only the groups of its episode's types.
#pragma once

#include <string>

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fem.h"

namespace fem {

constexpr uint32_t CHUNK = 2048;            // events per staged chunk
constexpr uint32_t KEY_END = 0xFFFFFFFFu;   // "list exhausted"
constexpr uint32_t CLS_NONE = 0xFFFFFFFFu;  // MapConcatenate class "no recent completion"
constexpr uint32_t CLS_EMPTY = 0xFFFFFFFEu; // unused transfer-table slot
constexpr int S_MAX = 8;                    // MapConcatenate entry classes per table
constexpr int S_RECOUNT = 32;               // the same, in the segmented recount

// device error word bits
constexpr uint32_t ERR_TIMEOUT = 1u;       // a bounded mbarrier wait gave up
constexpr uint32_t ERR_RING = 2u;          // an exact-pass list outgrew its ring (host retries)
constexpr uint32_t ERR_BADEP = 4u;         // malformed candidate (type/len/interval index)
constexpr uint32_t ERR_UNSORTED = 8u;
constexpr uint32_t ERR_TYPE = 16u;
constexpr uint32_t ERR_TABLE = 32u;        // transfer table missing a class (internal)
constexpr uint32_t ERR_CLASS = 64u;        // more entry classes than table slots (host retries)
constexpr uint32_t ERR_NODES = 128u;       // a latest-chain block's prefix tables overflowed (host retries)
// any capacity guard: the flagged episodes are recounted by the host
constexpr uint32_t ERR_CAP = ERR_RING | ERR_TABLE | ERR_CLASS | ERR_NODES;

constexpr uint64_t WAIT_NS = 2000000000ull; // bound on any single device wait (2 s)

__host__ __device__ inline uint32_t offs_stride(uint32_t K) { return (K + 1 + 7) & ~7u; }
__host__ __device__ inline uint32_t stage_bytes(uint32_t offs) {
    return (CHUNK * 8u + offs * 2u + 127u) & ~127u;
}

struct StreamDev {
    uint64_t cap_events = 0, cap_chunks = 0;  // allocated capacity (buffers are reused)
    uint32_t cap_offs = 0;
    uint64_t n = 0;
    uint32_t K = 0, n_chunks = 0, offs = 0;
    uint32_t t_max = 0;
    uint32_t *t = nullptr;
    uint8_t *type = nullptr;
    uint2 *bev = nullptr;
    uint16_t *boff = nullptr;
    uint32_t *cfirst = nullptr;
    uint32_t *hist = nullptr;
    uint64_t gen = 0;  // contents' generation: new at every load and append (cache key)
    // the ring choice for the last interval set counted over these contents (host side)
    mutable uint64_t ring_gen = 0;
    mutable std::string ring_ivl;
    mutable bool ring_singles = false, ring_clusters = false;
};

// Arguments of the counting kernels (one pass over one candidate set).
struct CountParams {
    const uint2 *bev;
    const uint16_t *boff;
    const uint32_t *cfirst;
    const uint32_t *t;          // event times (read only for MapConcatenate exits)
    uint32_t offs, n_chunks;
    uint64_t n;
    uint32_t K;
    const fem_episode *cands;   // candidate records
    const uint32_t *gather;     // optional: count cands[gather[i]] as candidate i
    uint32_t m;
    const uint2 *ivl;           // (lo, hi) table
    uint32_t n_ivl;
    uint32_t *out;              // counts [m] (single segment)
    uint32_t cps;               // chunks per segment
    uint32_t P;                 // segments
    uint4 *tables;              // [P][m][S_MAX] (key, count, exit, 0) when P > 1
    uint8_t *redo;              // [m] set to 1 when a candidate must be recounted
    uint32_t *err;
    // optional (per-thread machine kernels):
    const uint32_t *m_dev;      // candidate count read on the device (overrides m)
    uint32_t ranged;            // count events [ev_begin, ev_end) only (segments from its first chunk)
    uint64_t ev_begin, ev_end;
    // (single segment only)
    uint32_t *state;            // per-candidate carried state (count, machine), in and out
    uint32_t state_stride;      // words per candidate: 1 + (N-1) relaxed, 1 + (N-1)(1 + 2R) exact
    // (level-2 pair kernel) frequent types f of a level-2 set of f (f - 1) n_ivl candidates
    uint32_t pair_types;
};

// MapConcatenate as printed (fem_literal.cu): time segments (tau[p], tau[p+1]]
struct LiteralParams {
    const uint2 *bev;
    const uint16_t *boff;
    const uint32_t *t;
    uint32_t offs;
    uint64_t n;
    const fem_episode *cands;   // m records, distinct types
    uint32_t m;
    const uint2 *ivl;
    const int64_t *tau;         // P + 1 increasing times, tau[0] < t[0], tau[P] >= t[n-1]
    uint32_t P;
    uint4 *tuples;              // [m][P][FEM_MAX_LEN]
    uint32_t *err;
};

// Per-job output arrays of a batch (device pointers owned by the caller).
struct BatchOut {
    uint32_t *exact;
    uint8_t *survived;
};

// ---------------------------------------------------------------- PTX helpers
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared (TMA engine), completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of `bar`, giving up after WAIT_NS (sets ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t *err) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0 && global_ns() - t0 > WAIT_NS) {
            atomicOr(err, ERR_TIMEOUT);
            return false;
        }
    }
}
#endif

// ---------------------------------------------------------------- launchers (host side)
// process-wide count of kernel launches (fem_kernel_launches)
void note_launch(uint32_t k = 1);

// fem_stream.cu
// Validate and group a stream already in s.t / s.type, or (src_t given) one in other
// device memory, copying it into s.t / s.type on the way.
cudaError_t launch_load_stream(StreamDev &s, cudaStream_t st, uint32_t *d_err,
                               const uint32_t *src_t = nullptr, const uint8_t *src_type = nullptr);
// regroup chunks [c0, c1) of a stream that grew to s.n events (type histogram untouched);
// with d_err the chunks' events are also checked (types < K, times non-decreasing)
cudaError_t launch_bucket_chunks(StreamDev &s, uint32_t c0, uint32_t c1, cudaStream_t st,
                                 uint32_t *d_err = nullptr);
// hist[ty[i]] += sign (+1 or -1) for i < n
// host[0] = *err, host[1] = *t_last (0 if null), host[2 .. 2 + K) = hist, then
// host[seq_word] = seq (host: the device address of mapped pinned words)
cudaError_t launch_publish_load(const uint32_t *err, const uint32_t *t_last, const uint32_t *hist,
                                uint32_t K, uint32_t *host, uint32_t seq_word, uint32_t seq,
                                cudaStream_t st);
// fem_pairs.cu: the relaxed pass of a level-2 set, all interval variants of an ordered
// type pair in one thread (p.pair_types = f, p.n_ivl <= 4; P > 1: MapConcatenate tables)
cudaError_t launch_pairs_relaxed(const CountParams &p, uint32_t threads, cudaStream_t st);
size_t pairs_smem_bytes(bool mc, uint32_t threads, uint32_t offs);
// after that pass in level-wise mining: the flagged candidates' counts set to pass any
// threshold; their capacity bits cleared when at most `limit` are flagged (work: two
// words, zero before the first launch, left zero)
cudaError_t launch_pairs_pass_flagged(uint32_t *out, const uint8_t *redo, uint32_t m,
                                      uint32_t limit, uint32_t *work, uint32_t *err,
                                      cudaStream_t st);
// cap[a * nh + j] (zeroed by the caller): the most type-a events in a closed window of
// length h[j] (device array); with dense (zeroed), also the number of type-a events whose
// window of length h[j] holds more than `over` events
cudaError_t launch_capacity(const StreamDev &s, const uint32_t *h, uint32_t nh, uint32_t *cap,
                            cudaStream_t st, uint32_t over = 0, uint32_t *dense = nullptr);
cudaError_t launch_hist_add(const uint8_t *ty, uint64_t n, uint32_t K, int sign, uint32_t *hist,
                            cudaStream_t st);
// dst[idx[i]] = src[i] and flags[idx[i]] = 1 for i < *m_dev (grid sized for m_max)
cudaError_t launch_scatter_dev(const uint32_t *src, const uint32_t *idx, const uint32_t *m_dev,
                               uint32_t m_max, uint32_t *dst, uint8_t *flags, cudaStream_t st);
int fem_ctx_device(const fem_ctx *c);
int fem_ctx_sms(const fem_ctx *c);
// fem_count.cu
// classes: entry-class slots per transfer table (S_MAX; 2 S_MAX for the segmented recount,
// relaxed or exact with ring_cap 32)
cudaError_t launch_count(int N, int pass, bool mc, uint32_t ring_cap, uint32_t threads,
                         const CountParams &p, cudaStream_t st, uint32_t classes = S_MAX);
size_t count_smem_bytes(int N, int pass, bool mc, uint32_t ring_cap, uint32_t threads,
                        uint32_t offs, uint32_t classes = S_MAX);
bool count_config_supported(int N, int pass, bool mc, uint32_t ring_cap);
// persistent batched counting (segmented form for every job; ring_cap 8/16/32 for exact)
cudaError_t launch_count_batch(int N, int pass, uint32_t ring_cap, uint32_t threads,
                               const CountParams *jobs, const uint4 *items,
                               const uint32_t *n_items, uint32_t *queue, uint32_t SB,
                               int sm_count, cudaStream_t st);
cudaError_t count_set_smem_limits();
// fem_chain_*.cu: the same passes in latest-chain form (distinct types, lengths 2..8,
// one segment or MapConcatenate; candidates sharing prefixes share their lists)
cudaError_t launch_chain(int N, int pass, bool mc, uint32_t threads, const CountParams &p,
                         cudaStream_t st);
size_t chain_smem_bytes(int N, bool mc, uint32_t threads, uint32_t offs);
// fem_windows.cu: window-based frequency, one thread per episode (distinct types)
struct WindowParams {
    const uint2 *bev;
    const uint16_t *boff;
    uint32_t offs;
    uint64_t n;
    const fem_episode *cands;
    uint32_t m;
    const uint2 *ivl;
    uint32_t w;          // window width (us), > 0
    uint64_t *out;       // [m]
    uint32_t *err;
};
cudaError_t launch_count_windows(const WindowParams &p, uint32_t len_mask, cudaStream_t st);
// fem_literal.cu: map (one thread per episode, segment and machine) and join;
// len_mask has bit N set for every episode length N present; diag[2] accumulates the
// boundaries where no tuple / several tuples matched
cudaError_t launch_literal(const LiteralParams &p, uint32_t len_mask, uint32_t *out, uint32_t *diag,
                           cudaStream_t st);
// fem_mine.cu
// stitch of a batch: job_base[j] = first global episode slot of job j (n_jobs + 1
// entries); slots >= a job's current m are skipped
cudaError_t launch_stitch_batch(const CountParams *jobs, const uint32_t *job_base,
                                uint32_t n_jobs, uint32_t slots, uint32_t *err, cudaStream_t st);
cudaError_t launch_stitch(const uint4 *tables, uint32_t m, uint32_t P, uint32_t *out,
                          uint8_t *redo, uint32_t *err, cudaStream_t st,
                          uint32_t classes = S_MAX);
// info[0] |= 1 << len of every candidate; info[1] += candidates with a repeated type;
// info[2] += candidates whose length or prefix before the last node differs from the
// previous candidate's (the number of prefix runs is info[2] + 1)
cudaError_t launch_validate_cands(const fem_episode *c, const uint32_t *gather, uint32_t m,
                                  uint32_t K, uint32_t n_ivl, uint32_t *info, uint32_t *err,
                                  cudaStream_t st);
cudaError_t launch_len_flags(const fem_episode *c, const uint32_t *gather, uint32_t m, uint32_t N,
                             uint8_t *flags, cudaStream_t st);
// dst[i] = outer ? outer[inner[i]] : inner[i]
cudaError_t launch_touched(const fem_episode *cands, const uint32_t *gather, uint32_t m,
                           const uint32_t *hist, unsigned long long *out, cudaStream_t st);
cudaError_t launch_compose_idx(const uint32_t *outer, const uint32_t *inner, uint32_t m,
                               uint32_t *dst, cudaStream_t st);
// stable compaction: keep[i] = (vals[i] >= theta) (or flags[i] != 0 if vals == NULL)
// block_scratch holds compact_scratch_words(m) words: one partial sum per block of
// COMPACT_ITEMS_PER_BLOCK items plus a slack of 32
// A count a kernel also writes, with the error word, into pinned host memory (the device
// address of three mapped host words): count, error word, then -- after a system-wide
// fence -- the sequence number `seq`, which tells the host both words are there.
struct Publish {
    uint32_t *host = nullptr;
    const uint32_t *err = nullptr;
    uint32_t seq = 0;
};
cudaError_t launch_compact(const uint32_t *vals, const uint8_t *flags, uint32_t theta, uint32_t m,
                           uint32_t *idx_out, uint32_t *count_out, uint32_t *block_scratch,
                           cudaStream_t st, Publish pub = {});
constexpr uint32_t COMPACT_ITEMS_PER_BLOCK = 1024;
constexpr size_t compact_scratch_words_for(uint64_t m) {
    return (size_t)((m + COMPACT_ITEMS_PER_BLOCK - 1) / COMPACT_ITEMS_PER_BLOCK) + 32;
}
size_t compact_scratch_words(uint32_t m);
cudaError_t launch_gather_frequent(const fem_episode *cands, const uint32_t *surv,
                                   const uint32_t *idx, uint32_t f, const uint32_t *counts,
                                   fem_episode *F, uint32_t *fcnt, cudaStream_t st);
cudaError_t launch_gather_episodes(const fem_episode *src, const uint32_t *idx, uint32_t m,
                                   fem_episode *dst, const uint32_t *vals, uint32_t *vals_dst,
                                   cudaStream_t st);
cudaError_t launch_scatter_u32(const uint32_t *src, const uint32_t *idx, uint32_t m,
                               uint32_t *dst, cudaStream_t st);
cudaError_t launch_fill_flags(const uint32_t *idx, uint32_t m, uint8_t *flags, cudaStream_t st);
cudaError_t launch_level2(const uint32_t *ftypes, uint32_t f, uint32_t n_ivl, bool repeats,
                          fem_episode *out, cudaStream_t st);
cudaError_t launch_join_count(const fem_episode *F, uint32_t f, uint32_t N, bool repeats,
                              uint32_t *cnt, int sm_count, cudaStream_t st);
cudaError_t launch_exclusive_scan(const uint32_t *in, uint32_t m, uint32_t *out,
                                  uint32_t *total, uint32_t *scratch, cudaStream_t st,
                                  Publish pub = {});
cudaError_t launch_join_emit(const fem_episode *F, uint32_t f, uint32_t N, bool repeats,
                             const uint32_t *off, fem_episode *out, int sm_count, cudaStream_t st);
cudaError_t launch_repeat_flags(const fem_episode *c, const uint32_t *gather, uint32_t m, bool invert,
                                uint8_t *flags, cudaStream_t st);
// fem_batch.cu
cudaError_t launch_batch_items(const CountParams *jobs, uint32_t n_jobs, uint32_t T,
                               uint32_t *item_off, uint32_t *n_items, uint32_t cap, uint4 *items,
                               cudaStream_t st);
cudaError_t launch_batch_keep_flags(const uint32_t *rel, const uint32_t *cand_off,
                                    const uint32_t *theta, uint32_t n_jobs, uint32_t m,
                                    uint8_t *flags, cudaStream_t st);
cudaError_t launch_batch_exact_jobs(CountParams *xjobs, const uint32_t *cand_off, uint32_t n_jobs,
                                    const uint32_t *idx, const uint32_t *n_idx, uint32_t *ex,
                                    cudaStream_t st);
cudaError_t launch_batch_outputs(const BatchOut *outs, const uint32_t *cand_off, uint32_t n_jobs,
                                 uint32_t m, const uint32_t *idx, const uint32_t *n_idx,
                                 const uint32_t *ex, cudaStream_t st);
cudaError_t launch_type_filter(const uint32_t *hist, uint32_t K, uint32_t theta,
                               uint32_t *ftypes, uint32_t *fcount, cudaStream_t st);

}  // namespace fem
