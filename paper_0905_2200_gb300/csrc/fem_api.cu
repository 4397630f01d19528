// fem_api.cu -- the C ABI of libfem.so (include/fem.h): contexts, resident
// streams, the counting driver (segment choice, capacity retries), Algorithm 4
// and the level-wise miner of Problem 1.  Every step of the method runs in the
// kernels of fem_stream.cu, fem_count.cu and fem_mine.cu; this file only
// allocates device memory, launches, and copies results.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "fem_internal.cuh"

using namespace fem;

namespace fem {
static std::atomic<uint64_t> g_launches{0};
void note_launch(uint32_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace fem

struct fem_result {
    std::vector<std::vector<fem_episode>> eps;    // [level-1]
    std::vector<std::vector<uint32_t>> counts;  // [level-1]
};

namespace {
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};
}  // namespace

struct fem_ctx {
    int device = 0;
    // device memory the context holds for streams, working buffers and batches, and
    // the caller's bound on it (0: none)
    size_t mem_budget = 0, mem_used = 0;
    cudaStream_t own = nullptr;
    fem_config cfg{};
    int sm_count = 152;
    std::map<int32_t, StreamDev> streams;
    // per loaded stream, its type histogram (the level-1 counts), read back in the
    // load's own round trip so that mining needs no wait for it
    std::map<int32_t, std::vector<uint32_t>> hist_h;
    int32_t next_id = 1;
    uint32_t *d_err = nullptr;    // device error word
    uint32_t *d_small = nullptr;  // 64 device words for counters
    uint32_t *h_small = nullptr;  // 64 pinned host words
    // device address of h_small[kPubWord..kPubWord+1], written by the compaction and scan
    // kernels (count and error word); null where pinned memory is not mapped
    uint32_t *d_pub = nullptr;
    uint32_t pub_seq = 0;  // sequence number of the last publishing launch
    // mapped pinned words a load's read-back is published to ([0] error word, [1] last
    // time, [2..258) type counts, [kLoadSeq] sequence number) and their device address
    uint32_t *h_load = nullptr, *d_load = nullptr;
    // pinned staging of an interval set (so that its upload is asynchronous), and the
    // event after the last upload from it (the next one waits for that copy to leave)
    fem_interval *h_ivl = nullptr;
    cudaEvent_t ivl_ev = nullptr;
    std::vector<fem_interval> ivl_host;  // the interval set of the current call
    uint64_t next_gen = 1;  // stream contents' generations
    std::map<std::string, DevBuf> bufs;
    std::vector<fem_level_stats> stats;
    std::vector<StreamDev> pool;  // buffers of freed streams, reused by later loads
    // mining timings: [0,1] generation, [2,3] relaxed pass, [4,5] compaction, [6,7] exact
    cudaEvent_t ev[8] = {};
    // pinned host staging of each level's frequent set (copied out after the last sync)
    struct PinBuf {
        void *p = nullptr;
        size_t cap = 0;
    };
    PinBuf pin[FEM_MAX_LEN + 1];
    // around the counting kernel and stitch, two sets used in turn, so that a pass's
    // times can be read after the next pass has been queued
    cudaEvent_t kev[2][3] = {};
    int kev_flip = 0;
    // measured mapping choice: launch shape per (N, pass, distinct, log2 m,
    // log2 chunks, K) class
    struct Shape {
        uint32_t P, T;
        float ms;
        uint32_t kernel;  // FEM_KERNEL_MACHINE or FEM_KERNEL_CHAIN
    };
    std::map<std::string, Shape> tune;
    bool tune_on = false, tuning = false;
    // the candidate set being counted comes in runs of shared prefixes (mining's sets
    // always do; count_any measures it): where it does not, the latest-chain kernels
    // would find few prefixes to share
    bool clustered = true;
    cudaEvent_t tev[2] = {nullptr, nullptr};
};

namespace {

// FEM_DEBUG set: a failing CUDA call is reported on stderr with its line
void report_cuda(cudaError_t e, int line) {
    if (std::getenv("FEM_DEBUG"))
        std::fprintf(stderr, "fem: CUDA error %s at fem_api.cu:%d\n", cudaGetErrorString(e), line);
}
#define CK(x)                          \
    do {                               \
        cudaError_t e_ = (x);          \
        if (e_ != cudaSuccess) {       \
            report_cuda(e_, __LINE__); \
            return FEM_ECUDA;          \
        }                              \
    } while (0)
#define RET(x)                  \
    do {                        \
        int r_ = (x);           \
        if (r_ != FEM_OK) return r_; \
    } while (0)

// d_small word assignment
enum { W_COUNT0 = 0, W_COUNT1 = 1, W_COUNT2 = 2, W_INFO = 8 /* 3 words */ };
// first of the three pinned host words the kernels publish counts to
constexpr uint32_t kPubWord = 48;
constexpr uint32_t kLoadSeq = 2 + 256;  // the load read-back's sequence word

size_t stream_bytes(const StreamDev &s) {
    if (!s.t) return 0;
    return s.cap_events * 5 + s.cap_chunks * CHUNK * 8 + (size_t)s.cap_offs * 2 +
           (s.cap_chunks + 1) * 4 + 256 * 4;
}

void free_stream_buffers(StreamDev &s);

// Room for `bytes` more under the context's memory budget: over budget, the buffers
// kept from freed streams are released first; FEM_ENOMEM if it still does not fit.
int reserve(fem_ctx *c, size_t bytes) {
    if (!c->mem_budget) return FEM_OK;
    while (c->mem_used + bytes > c->mem_budget && !c->pool.empty()) {
        c->mem_used -= std::min(stream_bytes(c->pool.front()), c->mem_used);
        free_stream_buffers(c->pool.front());
        c->pool.erase(c->pool.begin());
    }
    return c->mem_used + bytes > c->mem_budget ? FEM_ENOMEM : FEM_OK;
}

// Device allocation charged to the context's memory budget.
int cmalloc(fem_ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    RET(reserve(c, bytes));
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return FEM_ENOMEM;
    }
    c->mem_used += bytes;
    return FEM_OK;
}

void cfree(fem_ctx *c, void *p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    c->mem_used -= std::min(bytes, c->mem_used);
}

template <typename T>
int dbuf(fem_ctx *c, const char *name, size_t count, T **out) {
    const size_t bytes = std::max<size_t>(count * sizeof(T), 256);
    DevBuf &b = c->bufs[name];
    if (b.cap < bytes) {
        size_t nb = std::max(bytes, (size_t)(b.cap * 3 / 2));
        cfree(c, b.p, b.cap);
        b.p = nullptr;
        b.cap = 0;
        nb = (nb + 4095) & ~(size_t)4095;
        RET(cmalloc(c, &b.p, nb));
        b.cap = nb;
    }
    *out = static_cast<T *>(b.p);
    return FEM_OK;
}

cudaStream_t pick(fem_ctx *c, void *s) { return s ? static_cast<cudaStream_t>(s) : c->own; }

// Pinned host buffer `slot` of at least `bytes` (contents are not kept on growth; the
// stream is drained first, so no copy into the old buffer is in flight).
int pinbuf(fem_ctx *c, uint32_t slot, size_t bytes, cudaStream_t st, void **out) {
    fem_ctx::PinBuf &b = c->pin[slot];
    if (b.cap < bytes) {
        CK(cudaStreamSynchronize(st));
        if (b.p) cudaFreeHost(b.p);
        b.p = nullptr;
        b.cap = 0;
        const size_t nb = (std::max(bytes, (size_t)4096) + 4095) & ~(size_t)4095;
        if (cudaMallocHost(&b.p, nb) != cudaSuccess) {
            cudaGetLastError();
            return FEM_ENOMEM;
        }
        b.cap = nb;
    }
    *out = b.p;
    return FEM_OK;
}

int read_words(fem_ctx *c, const uint32_t *d, uint32_t n, uint32_t *h, cudaStream_t st) {
    CK(cudaMemcpyAsync(c->h_small, d, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::memcpy(h, c->h_small, n * sizeof(uint32_t));
    return FEM_OK;
}

int read_err(fem_ctx *c, cudaStream_t st, uint32_t *err) {
    return read_words(c, c->d_err, 1, err, st);
}

// The count (and error word) the next compaction or scan publishes into the mapped host
// words, under a new sequence number.
Publish pub_of(fem_ctx *c) {
    if (!c->d_pub) return Publish{};
    return Publish{c->d_pub, c->d_err, ++c->pub_seq};
}

// Wait until the mapped word `w` holds `seq` (written by a kernel on st after what it
// publishes): the host watches the word rather than waiting for the stream, so it can
// queue the next launches while that kernel retires; after 2 s it waits for the stream.
int wait_seq(const volatile uint32_t *w, uint32_t seq, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    for (uint32_t spin = 1; *w != seq; ++spin) {
        if ((spin & 1023u) == 0 && std::chrono::steady_clock::now() - t0 > std::chrono::seconds(2)) {
            CK(cudaStreamSynchronize(st));
            if (*w != seq) return FEM_ECUDA;
            break;
        }
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    return FEM_OK;
}

// A device count and the error word, in one round trip: read from the mapped words once
// the launch before has published them under its sequence number, else copied.
int read_count_err(fem_ctx *c, const uint32_t *d_count, uint32_t *count, uint32_t *err,
                   cudaStream_t st) {
    if (c->d_pub) {
        const volatile uint32_t *h = c->h_small + kPubWord;
        RET(wait_seq(h + 2, c->pub_seq, st));
        *count = h[0];
        *err = h[1];
        return FEM_OK;
    }
    CK(cudaMemcpyAsync(c->h_small, d_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(c->h_small + 1, c->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *count = c->h_small[0];
    *err = c->h_small[1];
    return FEM_OK;
}

int err_status(uint32_t e) {
    if (e & ERR_TIMEOUT) return FEM_ETIMEOUT;
    if (e & ERR_BADEP) return FEM_EINVAL;
    if (e & ERR_TYPE) return FEM_ETYPE;
    if (e & ERR_UNSORTED) return FEM_EUNSORTED;
    return FEM_OK;
}

const StreamDev *find_stream(fem_ctx *c, int32_t id) {
    auto it = c->streams.find(id);
    return it == c->streams.end() ? nullptr : &it->second;
}

int check_intervals(const StreamDev &s, const fem_interval *I, uint32_t nI) {
    if (nI > FEM_MAX_INTERVALS) return FEM_EINVAL;
    if (nI && !I) return FEM_EINVAL;
    uint64_t max_hi = 0;
    for (uint32_t i = 0; i < nI; ++i) {
        if (I[i].lo_us >= I[i].hi_us) return FEM_EINVAL;
        max_hi = std::max<uint64_t>(max_hi, I[i].hi_us);
    }
    // deadlines t + hi + 1 must fit in 32 bits
    if ((uint64_t)s.t_max + max_hi + 1 > 0xFFFFFFFFull) return FEM_ERANGE;
    return FEM_OK;
}

int upload_intervals(fem_ctx *c, const fem_interval *I, uint32_t nI, cudaStream_t st,
                     uint2 **d_ivl) {
    RET(dbuf(c, "ivl", std::max<uint32_t>(nI, 1), d_ivl));
    c->ivl_host.assign(I, I + nI);
    if (!nI) return FEM_OK;
    if (nI > FEM_MAX_INTERVALS + 1) {
        CK(cudaMemcpyAsync(*d_ivl, I, nI * sizeof(uint2), cudaMemcpyHostToDevice, st));
        return FEM_OK;
    }
    CK(cudaEventSynchronize(c->ivl_ev));  // the previous upload has left the staging
    std::memcpy(c->h_ivl, I, nI * sizeof(fem_interval));
    CK(cudaMemcpyAsync(*d_ivl, c->h_ivl, nI * sizeof(uint2), cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(c->ivl_ev, st));
    return FEM_OK;
}

// Capacity table of a resident stream for the given widths (host out[a * nh + j]);
// synchronous on st.  A width >= the stream's last time holds every event of a type.
// With dense_out (uint32[K * nh]): also the events of each type whose window of each width
// holds more than `over` events of the type.
int capacity(fem_ctx *c, const StreamDev &s, const uint32_t *widths, uint32_t nh,
             uint32_t *out, cudaStream_t st, uint32_t over = 0, uint32_t *dense_out = nullptr) {
    const uint32_t K = s.K;
    std::vector<uint32_t> hw, slot;
    for (uint32_t j = 0; j < nh; ++j)
        if (s.n && widths[j] < s.t_max) hw.push_back(widths[j]), slot.push_back(j);
    std::vector<uint32_t> hist(K, 0), part((size_t)K * hw.size(), 0), dpart(part.size(), 0);
    CK(cudaMemcpyAsync(hist.data(), s.hist, K * 4, cudaMemcpyDeviceToHost, st));
    if (!hw.empty()) {
        const uint32_t nk = (uint32_t)hw.size();
        uint32_t *d;
        RET(dbuf(c, "cap", (size_t)nk * (2 * K + 1), &d));
        uint32_t *d_dense = d + (size_t)K * nk, *d_h = d + (size_t)2 * K * nk;
        CK(cudaMemsetAsync(d, 0, (size_t)2 * K * nk * 4, st));
        CK(cudaMemcpyAsync(d_h, hw.data(), nk * 4, cudaMemcpyHostToDevice, st));
        CK(launch_capacity(s, d_h, nk, d, st, over, dense_out ? d_dense : nullptr));
        CK(cudaMemcpyAsync(part.data(), d, (size_t)K * nk * 4, cudaMemcpyDeviceToHost, st));
        if (dense_out)
            CK(cudaMemcpyAsync(dpart.data(), d_dense, (size_t)K * nk * 4, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    for (uint32_t a = 0; a < K; ++a) {
        for (uint32_t j = 0; j < nh; ++j) {
            out[(size_t)a * nh + j] = hist[a];
            if (dense_out) dense_out[(size_t)a * nh + j] = hist[a] > over ? hist[a] : 0u;
        }
        for (size_t q = 0; q < hw.size(); ++q) {
            out[(size_t)a * nh + slot[q]] = part[a * hw.size() + q];
            if (dense_out) dense_out[(size_t)a * nh + slot[q]] = dpart[a * hw.size() + q];
        }
    }
    return FEM_OK;
}

// Whether the per-thread exact kernel's lists should get rings of 32 entries instead of 8
// for the current interval set, from the capacity table: Algorithm 1's pruned list for
// node k holds type-E_k events within hi_k, as single times at most cap[E_k][hi_k] of
// them, as clusters at most ceil(hi / (hi - lo)) + 1.  Larger rings cost occupancy, so
// they are taken only where lists outgrow 8 often: more than one event in a thousand
// starts a window of length hi holding more than 8 events of its type (a bursting
// recording: 7% at 20 ms; an hour of 50 Hz Poisson trains: 0.001%, where the few
// episodes that overflow are recounted).  Kept with the stream for its contents and the
// last interval set.
constexpr uint32_t kRingSmall = 8, kRingLarge = 32;
int ring_choice(fem_ctx *c, const StreamDev &s, bool *large_singles, bool *large_clusters,
                cudaStream_t st) {
    const std::vector<fem_interval> &I = c->ivl_host;
    const std::string key(reinterpret_cast<const char *>(I.data()), I.size() * sizeof(fem_interval));
    if (s.ring_gen != s.gen || s.ring_ivl != key) {
        std::vector<uint32_t> w;
        for (const fem_interval &iv : I) w.push_back(iv.hi_us);
        std::vector<uint32_t> cap((size_t)s.K * w.size()), dense(cap.size());
        bool sg = false, cl = false;
        if (!w.empty() && s.n) {
            RET(capacity(c, s, w.data(), (uint32_t)w.size(), cap.data(), st, kRingSmall,
                         dense.data()));
            for (size_t j = 0; j < w.size(); ++j) {
                uint32_t mx = 0;
                uint64_t nd = 0;
                for (uint32_t a = 0; a < s.K; ++a) {
                    mx = std::max(mx, cap[(size_t)a * w.size() + j]);
                    nd += dense[(size_t)a * w.size() + j];
                }
                const bool often = nd * 1000 > s.n;
                const uint32_t span = I[j].hi_us - I[j].lo_us;
                const uint32_t ncl = (I[j].hi_us + span - 1) / span + 1;
                sg = sg || (often && mx > kRingSmall);
                cl = cl || (often && std::min(mx, ncl) > kRingSmall);
            }
        }
        s.ring_gen = s.gen;
        s.ring_ivl = key;
        s.ring_singles = sg;
        s.ring_clusters = cl;
    }
    *large_singles = s.ring_singles;
    *large_clusters = s.ring_clusters;
    return FEM_OK;
}

// Segments per episode for one pass.  One thread per (episode, segment); the aim is
// about 2048 threads per SM, and about 1024 for the two-node latest-chain kernel (one
// resident wave of its four 256-thread blocks per SM): the shapes the tuner keeps on
// the 64-type recording -- level-2 exact 29 segments (0.169 ms where 50 took 0.201),
// 13 on the deep variant -- while its longer episodes keep the larger aim (level-4
// exact of the deep variant: 6 segments 1.65 ms, 3 took 2.07).  Segments are whole
// chunks, so at most one per chunk.
uint32_t choose_segments(fem_ctx *c, const StreamDev &s, uint32_t m, bool distinct,
                         bool one_wave = false) {
    if (s.n_chunks == 0) return 1;
    const uint32_t maxP = std::min<uint32_t>(s.n_chunks, 65535);
    if (c->cfg.segments) return std::min<uint32_t>(c->cfg.segments, s.n_chunks);
    if (!distinct) return 1;
    const uint64_t target = (uint64_t)c->sm_count * (one_wave ? 1024 : 2048);
    uint64_t P = (target + m - 1) / m;
    if (P < 2) return 1;
    return (uint32_t)std::min<uint64_t>(P, maxP);
}

// Block size by shared memory (and, for few episodes, smaller blocks), ignoring any
// configured size.
uint32_t auto_threads(int N, int pass, bool mc, uint32_t R, uint32_t offs, uint32_t m,
                      uint32_t classes = S_MAX) {
    for (uint32_t T : {256u, 128u, 64u, 32u}) {
        if (T > 32 && m <= T / 2) continue;  // few episodes: small blocks, more of them
        if (T == 256 && N > 3) continue;  // register budget
        if (count_smem_bytes(N, pass, mc, R, T, offs, classes) <= 80 * 1024) return T;
    }
    for (uint32_t T : {32u, 16u, 8u}) {
        if (count_smem_bytes(N, pass, mc, R, T, offs, classes) <= 220 * 1024) return T;
    }
    return 8;
}

uint32_t choose_threads(fem_ctx *c, int N, int pass, bool mc, uint32_t R, uint32_t offs,
                        uint32_t m) {
    if (c->cfg.threads_per_block) return c->cfg.threads_per_block;
    return auto_threads(N, pass, mc, R, offs, m);
}

struct PassInfo {
    uint32_t segments = 1;
    uint32_t kernel = 0;  // FEM_KERNEL_MACHINE or FEM_KERNEL_CHAIN
    float ms_kernel = 0, ms_stitch = 0;
};

uint32_t ceil_log2(uint64_t v) {
    uint32_t r = 0;
    while ((1ull << r) < v) ++r;
    return r;
}

// The latest-chain kernels count distinct-type episodes of 2..8 nodes in sets that come
// in runs of shared prefixes (level-wise mining's candidates; fem_count_candidates
// measures the runs).  (Scattered candidates would be counted in parts, one per run of
// the node tables' capacity: slower than the per-thread machine.)
constexpr uint32_t kChainSmallSet = 64;
bool chain_eligible(const fem_ctx *c, int N, bool distinct, uint32_t m) {
    return distinct && N >= 2 && N <= FEM_MAX_LEN && m > 0 && c->clustered;
}

// The rule's kernel where no measurement says otherwise.  The latest-chain kernels for
// the exact pass, whose per-thread machine (sliding-window lists) costs the most per
// event, over at least a block of candidates, or over a small set (there a block's eight
// warps build the prefix lists together where the per-thread machine leaves a single
// warp per block: level-3 exact of 32 survivors 0.097 -> 0.063 ms).  For the relaxed pass,
// whose single slot per node makes the per-thread machine cheap, the latest-chain kernels
// only for longer episodes in large sets, where many candidates share each prefix list
// (the deep variant of the 64-type recording: level 3, 2.4M candidates, 55.5 -> 32.0 ms;
// level 4, 73k, 3.65 -> 1.60 ms), or in small sets; at the bench step's 13,657 level-3
// candidates, many of them in short prefix runs, the two measured level.
constexpr uint32_t kChainLargeSet = 32768;
uint32_t rule_kernel(const fem_ctx *c, int N, int pass, bool distinct, uint32_t m) {
    if (!chain_eligible(c, N, distinct, m)) return FEM_KERNEL_MACHINE;
    if (pass == FEM_PASS_EXACT)
        return m >= 256 || m <= kChainSmallSet ? FEM_KERNEL_CHAIN : FEM_KERNEL_MACHINE;
    return N >= 3 && (m >= kChainLargeSet || m <= kChainSmallSet) ? FEM_KERNEL_CHAIN
                                                                   : FEM_KERNEL_MACHINE;
}

// Block size of the latest-chain kernels: 256 threads, also for a few episodes (the
// block's warps share the prefix-list builds).
uint32_t chain_threads(uint32_t) { return 256u; }

// The class a measured launch shape is kept for: counts of the same length,
// pass and type structure, with m and the stream length in the same power-of-two
// range and the same type count, map alike.
std::string tune_key(int N, int pass, bool distinct, uint32_t m, uint32_t n_chunks, uint32_t K) {
    char b[96];
    std::snprintf(b, sizeof(b), "%d/%d/%d/%u/%u/%u", N, pass, distinct ? 1 : 0, ceil_log2(m),
                  ceil_log2(n_chunks), K);
    return b;
}

int count_pass(fem_ctx *c, const StreamDev &s, const fem_episode *cands, const uint32_t *gather,
               uint32_t m, int N, const uint2 *d_ivl, uint32_t nI, int pass, uint32_t *out,
               bool distinct, cudaStream_t st, PassInfo *info);

// Mapping choice by measurement (it replaces the fixed crossover rule of
// Algorithm 2): time the rule's launch shape and its neighbours (half and twice
// the segments per episode, the other block size) on the real inputs and keep the
// fastest for the class.  Every trial is a complete, correct count.
int tune_pass(fem_ctx *c, const std::string &key, const StreamDev &s, const fem_episode *cands,
              const uint32_t *gather, uint32_t m, int N, const uint2 *d_ivl, uint32_t nI,
              int pass, uint32_t *out, bool distinct, cudaStream_t st) {
    // per kernel: its rule's segments, half and twice as many
    auto segment_choices = [&](bool chain_kind) {
        const uint32_t P0 = choose_segments(c, s, m, distinct, chain_kind && N == 2);
        std::vector<uint32_t> Ps{P0};
        if (distinct) {
            if (P0 > 1) Ps.push_back(std::max<uint32_t>(1, P0 / 2));
            if (P0 * 2 <= s.n_chunks) Ps.push_back(P0 * 2);
        }
        return Ps;
    };
    const uint32_t R0 = pass == FEM_PASS_EXACT ? (c->cfg.ring_capacity ? c->cfg.ring_capacity : 8) : 1;
    // the shapes to time: per segment count and kernel the rule's block size and its
    // neighbours; the rule's own shape first
    const bool chain = chain_eligible(c, N, distinct, m);
    const uint32_t k0 = c->cfg.kernel ? c->cfg.kernel : rule_kernel(c, N, pass, distinct, m);
    std::vector<fem_ctx::Shape> shapes;
    for (uint32_t kind : {k0, k0 == FEM_KERNEL_CHAIN ? (uint32_t)FEM_KERNEL_MACHINE : (uint32_t)FEM_KERNEL_CHAIN}) {
        if (kind == FEM_KERNEL_CHAIN && !chain) continue;
        if (c->cfg.kernel && kind != c->cfg.kernel) continue;
        for (uint32_t P : segment_choices(kind == FEM_KERNEL_CHAIN)) {
            if (kind == FEM_KERNEL_CHAIN) {
                const uint32_t T0 = chain_threads(m);
                shapes.push_back(fem_ctx::Shape{P, T0, -1.f, kind});
                for (uint32_t T : {128u, 256u})
                    if (T != T0 && m > T / 2 && chain_smem_bytes(N, P > 1, T, s.offs) <= 200 * 1024)
                        shapes.push_back(fem_ctx::Shape{P, T, -1.f, kind});
                continue;
            }
            const uint32_t R = (P > 1 && R0 > 32) ? 32 : R0;
            const uint32_t T0 = choose_threads(c, N, pass, P > 1, R, s.offs, m);
            shapes.push_back(fem_ctx::Shape{P, T0, -1.f, kind});
            for (uint32_t T : {128u, 256u})
                if (T != T0 && m > T / 2 && count_smem_bytes(N, pass, P > 1, R, T, s.offs) <= 100 * 1024)
                    shapes.push_back(fem_ctx::Shape{P, T, -1.f, kind});
        }
    }
    const fem_config saved = c->cfg;
    c->tuning = true;
    int rc = FEM_OK;
    // Two sweeps over all shapes, keeping each shape's faster time: interleaving keeps
    // a clock that is still rising at the first trials (or the first launch of a
    // kernel, which also loads it) from favouring the shapes timed last.
    for (int rep = 0; rep < 2 && rc == FEM_OK; ++rep) {
        for (fem_ctx::Shape &sh : shapes) {
            c->cfg.segments = sh.P;
            c->cfg.threads_per_block = sh.T;
            c->cfg.kernel = sh.kernel;
            cudaEventRecord(c->tev[0], st);
            rc = count_pass(c, s, cands, gather, m, N, d_ivl, nI, pass, out, distinct, st, nullptr);
            cudaEventRecord(c->tev[1], st);
            if (rc != FEM_OK) break;
            float t = 0;
            if (cudaEventSynchronize(c->tev[1]) != cudaSuccess ||
                cudaEventElapsedTime(&t, c->tev[0], c->tev[1]) != cudaSuccess) {
                rc = FEM_ECUDA;
                break;
            }
            if (sh.ms < 0 || t < sh.ms) sh.ms = t;
        }
    }
    // the rule's shape (the first) stays unless another is at least 2% faster
    fem_ctx::Shape best{0, 0, 0, 0};
    if (rc == FEM_OK && !shapes.empty()) {
        best = shapes[0];
        for (const fem_ctx::Shape &sh : shapes)
            if (sh.ms < 0.98f * best.ms) best = sh;
    }
    c->cfg = saved;
    c->tuning = false;
    if (rc == FEM_OK && best.P) c->tune[key] = best;
    return rc;
}

// A counting pass that has been launched: what its completion check needs.
struct PassLaunch {
    CountParams p{};
    int N = 0, pass = 0;
    bool distinct = true, chain = false;
    uint32_t R = 1;
    int evset = 0;  // the kernel event set recorded around it
    bool pairs = false;  // the level-2 pair kernel
};

// Launch one counting pass over m candidates (all of length N) -> out[0..m)
// (kernel, then the stitch when segmented), without waiting for it.  The pass is
// complete only after count_finish has seen the error word.
int count_launch(fem_ctx *c, const StreamDev &s, const fem_episode *cands, const uint32_t *gather,
                 uint32_t m, int N, const uint2 *d_ivl, uint32_t nI, int pass, uint32_t *out,
                 bool distinct, cudaStream_t st, PassLaunch *pl) {
    pl->p = CountParams{};
    pl->N = N, pl->pass = pass, pl->distinct = distinct;
    if (m == 0) return FEM_OK;
    // a measured shape for this class, if any (explicit configuration wins)
    uint32_t P_t = 0, T_t = 0, K_t = 0;
    if (!c->cfg.segments && !c->cfg.threads_per_block && !c->cfg.kernel && !c->tuning) {
        const std::string key = tune_key(N, pass, distinct, m, s.n_chunks, s.K);
        auto it = c->tune.find(key);
        if (it == c->tune.end() && c->tune_on) {
            RET(tune_pass(c, key, s, cands, gather, m, N, d_ivl, nI, pass, out, distinct, st));
            it = c->tune.find(key);
        }
        if (it != c->tune.end()) P_t = it->second.P, T_t = it->second.T, K_t = it->second.kernel;
    }
    uint32_t kind = c->cfg.kernel ? c->cfg.kernel : K_t;
    if (!kind) kind = rule_kernel(c, N, pass, distinct, m);
    // (a configured or cached choice of the latest-chain kernels needs distinct types only)
    if (kind == FEM_KERNEL_CHAIN && !(distinct && N >= 2)) kind = FEM_KERNEL_MACHINE;
    CountParams p{};
    p.bev = s.bev;
    p.boff = s.boff;
    p.cfirst = s.cfirst;
    p.t = s.t;
    p.offs = s.offs;
    p.n_chunks = s.n_chunks;
    p.n = s.n;
    p.K = s.K;
    p.cands = cands;
    p.gather = gather;
    p.m = m;
    p.ivl = d_ivl;
    p.n_ivl = nI;
    p.out = out;
    p.err = c->d_err;
    uint8_t *redo;
    RET(dbuf(c, "redo", m, &redo));
    CK(cudaMemsetAsync(redo, 0, m, st));
    p.redo = redo;

    uint32_t P = P_t ? std::min<uint32_t>(P_t, std::max<uint32_t>(s.n_chunks, 1))
                     : choose_segments(c, s, m, distinct, kind == FEM_KERNEL_CHAIN && N == 2);
    if (!distinct) P = 1;
    uint32_t R = 1;
    if (pass == FEM_PASS_EXACT) R = c->cfg.ring_capacity ? c->cfg.ring_capacity : 8;
    if (pass == FEM_PASS_EXACT && !c->cfg.ring_capacity && kind == FEM_KERNEL_MACHINE) {
        // rings sized from the capacity table where lists outgrow the small rings often
        // (bursting recordings), so that the first count does not overflow
        bool sg, cl;
        RET(ring_choice(c, s, &sg, &cl, st));
        if (P > 1 ? sg : cl) R = kRingLarge;
    }
    if (P > 1 && pass == FEM_PASS_EXACT && R > 32) R = 32;
    if (!count_config_supported(N, pass, P > 1, R)) return FEM_EINVAL;
    const uint32_t cps = P > 1 ? (s.n_chunks + P - 1) / P : std::max<uint32_t>(s.n_chunks, 1);
    if (P > 1) P = (s.n_chunks + cps - 1) / cps;
    p.cps = cps;
    p.P = P;
    if (P > 1) {
        RET(dbuf(c, "tables", (size_t)P * m * S_MAX, &p.tables));
    }
    const int es = c->kev_flip ^= 1;
    pl->evset = es;
    cudaEvent_t *kev = c->kev[es];
    CK(cudaEventRecord(kev[0], st));
    pl->chain = kind == FEM_KERNEL_CHAIN;
    if (kind == FEM_KERNEL_CHAIN) {
        uint32_t T = c->cfg.threads_per_block ? c->cfg.threads_per_block : (T_t ? T_t : chain_threads(m));
        if (chain_smem_bytes(N, P > 1, T, s.offs) > 200 * 1024) T = 128;
        CK(launch_chain(N, pass, P > 1, T, p, st));
    } else {
        uint32_t T = choose_threads(c, N, pass, P > 1, R, s.offs, m);
        if (T_t && count_smem_bytes(N, pass, P > 1, R, T_t, s.offs) <= 100 * 1024) T = T_t;
        // a configured block size whose rings would not fit in shared memory is replaced
        if (count_smem_bytes(N, pass, P > 1, R, T, s.offs) > 200 * 1024)
            T = auto_threads(N, pass, P > 1, R, s.offs, m);
        CK(launch_count(N, pass, P > 1, R, T, p, st));
    }
    CK(cudaEventRecord(kev[1], st));
    if (P > 1) CK(launch_stitch(p.tables, m, P, out, redo, c->d_err, st));
    CK(cudaEventRecord(kev[2], st));
    pl->p = p;
    pl->R = R;
    return FEM_OK;
}

// The relaxed pass of fem_mine_levelwise's level 2 (f frequent types x nI <= 4 intervals,
// m = f (f - 1) nI candidates in canonical order) with every interval variant of an
// ordered type pair in one thread (fem_pairs.cu); segments for about three 256-thread
// blocks per SM (or the configured count), tables, stitch and completion as in
// count_launch.
int count_launch_pairs(fem_ctx *c, const StreamDev &s, const fem_episode *cands, uint32_t m,
                       uint32_t f, const uint2 *d_ivl, uint32_t nI, uint32_t *out, cudaStream_t st,
                       PassLaunch *pl) {
    pl->p = CountParams{};
    pl->N = 2, pl->pass = FEM_PASS_RELAXED, pl->distinct = true, pl->chain = false;
    pl->pairs = true;
    if (m == 0) return FEM_OK;
    CountParams p{};
    p.bev = s.bev;
    p.boff = s.boff;
    p.cfirst = s.cfirst;
    p.t = s.t;
    p.offs = s.offs;
    p.n_chunks = s.n_chunks;
    p.n = s.n;
    p.K = s.K;
    p.cands = cands;
    p.m = m;
    p.ivl = d_ivl;
    p.n_ivl = nI;
    p.out = out;
    p.err = c->d_err;
    p.pair_types = f;
    uint8_t *redo;
    RET(dbuf(c, "redo", m, &redo));
    CK(cudaMemsetAsync(redo, 0, m, st));
    p.redo = redo;
    const uint64_t pairs = (uint64_t)f * (f - 1);
    uint32_t P;
    if (c->cfg.segments) {
        P = std::min<uint32_t>(c->cfg.segments, std::max<uint32_t>(s.n_chunks, 1));
    } else {
        const uint64_t target = (uint64_t)c->sm_count * 3 * 256;
        P = (uint32_t)std::min<uint64_t>((target + pairs - 1) / pairs, std::max<uint32_t>(s.n_chunks, 1));
    }
    const uint32_t cps = P > 1 ? (s.n_chunks + P - 1) / P : std::max<uint32_t>(s.n_chunks, 1);
    if (P > 1) P = (s.n_chunks + cps - 1) / cps;
    p.cps = cps;
    p.P = P;
    if (P > 1) RET(dbuf(c, "tables", (size_t)P * m * S_MAX, &p.tables));
    const int es = c->kev_flip ^= 1;
    pl->evset = es;
    cudaEvent_t *kev = c->kev[es];
    CK(cudaEventRecord(kev[0], st));
    CK(launch_pairs_relaxed(p, 256, st));
    CK(cudaEventRecord(kev[1], st));
    if (P > 1) CK(launch_stitch(p.tables, m, P, out, redo, c->d_err, st));
    CK(cudaEventRecord(kev[2], st));
    pl->p = p;
    pl->R = 1;
    return FEM_OK;
}

// Kernel and stitch times of the last launched pass (its events have completed).
void pass_info(fem_ctx *c, const PassLaunch &pl, PassInfo *info) {
    info->segments = pl.p.m ? pl.p.P : 0;
    info->kernel = pl.p.m ? (pl.pairs ? FEM_KERNEL_PAIRS
                                      : pl.chain ? FEM_KERNEL_CHAIN : FEM_KERNEL_MACHINE)
                          : 0u;
    info->ms_kernel = info->ms_stitch = 0;
    if (!pl.p.m) return;
    cudaEventElapsedTime(&info->ms_kernel, c->kev[pl.evset][0], c->kev[pl.evset][1]);
    cudaEventElapsedTime(&info->ms_stitch, c->kev[pl.evset][1], c->kev[pl.evset][2]);
}

// Complete a launched pass given the error word read after it: report hard errors,
// and recount the episodes whose rings or class tables overflowed.
int count_finish(fem_ctx *c, const StreamDev &s, const PassLaunch &pl, uint32_t e,
                 cudaStream_t st) {
    RET(err_status(e));
    if (!pl.p.m || !(e & ERR_CAP)) return FEM_OK;
    const CountParams &p = pl.p;
    const uint32_t m = p.m, P = p.P, R = pl.R;
    const int N = pl.N, pass = pl.pass;
    const bool distinct = pl.distinct;
    const uint32_t *gather = p.gather;
    uint32_t *out = p.out;
    uint8_t *redo = p.redo;

    // Recount the flagged episodes with one segment and larger rings.
    uint32_t *ridx, *rg, *rout, *scratch;
    RET(dbuf(c, "redo_idx", m, &ridx));
    RET(dbuf(c, "redo_scratch", compact_scratch_words(m), &scratch));
    CK(launch_compact(nullptr, redo, 0, m, ridx, c->d_small + W_COUNT2, scratch, st, pub_of(c)));
    uint32_t r, er;
    RET(read_count_err(c, c->d_small + W_COUNT2, &r, &er, st));
    if (std::getenv("FEM_DEBUG"))
        std::fprintf(stderr, "fem: pass %d N=%d m=%u P=%u R=%u: %u episodes recounted (err %#x)\n",
                     pass, N, m, P, R, r, e);
    if (r == 0) return FEM_OK;
    RET(dbuf(c, "redo_gather", r, &rg));
    RET(dbuf(c, "redo_out", r, &rout));
    CK(launch_compose_idx(gather, ridx, r, rg, st));
    // Episodes a latest-chain launch gave up on (its prefix tables or four class slots
    // were too small) go first to the per-thread kernels with the pass's own segments.
    // Then: the flagged episodes alone, one chunk per segment (short items, so the retry
    // costs about one chunk of work) with the largest segmented rings; last resort, one
    // segment per episode with the largest rings.
    struct Try {
        bool mc;
        uint32_t R;
        bool same_segments;
        uint32_t cls;  // entry-class slots of the segmented tables
    };
    std::vector<Try> tries;
    if (pl.pairs) tries.push_back({true, 8u, false, S_MAX});  // one chunk per segment
    if (pl.chain) {
        // a latest-chain launch that only ran out of its entry-class slots: the per-thread
        // kernel has twice the slots and merges classes before refusing one; one chunk per
        // segment, so that the few episodes spread over the GPU.  Other guards: the
        // per-thread kernel with the pass's own segments.
        if (e & ~ERR_CLASS & ERR_CAP) tries.push_back({P > 1, 8u, true, S_MAX});
        else tries.push_back({true, 8u, false, S_MAX});
    }
    tries.push_back({true, 32u, false, S_RECOUNT});  // four times the slots, larger rings
    tries.push_back({false, 32u, false, S_MAX});
    tries.push_back({false, 128u, false, S_MAX});
    for (const Try &tr : tries) {
        if (tr.mc && !distinct) continue;
        CK(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), st));
        CountParams q = p;
        q.gather = rg;
        q.m = r;
        q.out = rout;
        RET(dbuf(c, "redo2", r, &q.redo));
        CK(cudaMemsetAsync(q.redo, 0, r, st));
        const uint32_t Rq = pass == FEM_PASS_EXACT ? tr.R : 1;
        const uint32_t cls = tr.mc && s.n_chunks > 1 ? tr.cls : S_MAX;
        if (tr.same_segments) {
            if (q.P > 1) RET(dbuf(c, "redo_tables", (size_t)q.P * r * cls, &q.tables));
        } else if (tr.mc && s.n_chunks > 1) {
            q.P = s.n_chunks;
            q.cps = 1;
            RET(dbuf(c, "redo_tables", (size_t)q.P * r * cls, &q.tables));
        } else {
            q.P = 1;
            q.cps = std::max<uint32_t>(s.n_chunks, 1);
            q.tables = nullptr;
        }
        const bool mc2 = q.P > 1;
        // the recount's rings are larger: its block size is chosen for them, whatever
        // size is configured (or being tried) for the first count
        const uint32_t T2 = auto_threads(N, pass, mc2, Rq, s.offs, r, cls);
        CK(launch_count(N, pass, mc2, Rq, T2, q, st, cls));
        if (mc2) CK(launch_stitch(q.tables, r, q.P, rout, q.redo, c->d_err, st, cls));
        RET(read_err(c, st, &e));
        RET(err_status(e));
        if (std::getenv("FEM_DEBUG"))
            std::fprintf(stderr, "fem:   retry P=%u R=%u: err %#x\n", q.P, Rq, e);
        if (!(e & ERR_CAP)) {
            CK(launch_scatter_u32(rout, ridx, r, out, st));
            return FEM_OK;
        }
    }
    return FEM_EOVERFLOW;
}

// One counting pass, waited for and completed.
int count_pass(fem_ctx *c, const StreamDev &s, const fem_episode *cands, const uint32_t *gather,
               uint32_t m, int N, const uint2 *d_ivl, uint32_t nI, int pass, uint32_t *out,
               bool distinct, cudaStream_t st, PassInfo *info) {
    if (m == 0) return FEM_OK;
    PassLaunch pl;
    RET(count_launch(c, s, cands, gather, m, N, d_ivl, nI, pass, out, distinct, st, &pl));
    uint32_t e;
    RET(read_err(c, st, &e));
    if (info) pass_info(c, pl, info);
    return count_finish(c, s, pl, e, st);
}

// Validate a candidate set (optionally gathered) and count it with `pass`,
// grouping candidates by length.  out[i] is the count of candidate i of the
// (gathered) set.
int count_any(fem_ctx *c, const StreamDev &s, const fem_episode *cands, const uint32_t *gather,
              uint32_t m, const uint2 *d_ivl, uint32_t nI, int pass, uint32_t *out,
              cudaStream_t st) {
    if (m == 0) return FEM_OK;
    CK(cudaMemsetAsync(c->d_small + W_INFO, 0, 3 * sizeof(uint32_t), st));
    CK(launch_validate_cands(cands, gather, m, s.K, nI, c->d_small + W_INFO, c->d_err, st));
    uint32_t info[3], e;
    RET(read_words(c, c->d_small + W_INFO, 3, info, st));
    RET(read_err(c, st, &e));
    RET(err_status(e));
    const uint32_t lens = info[0];
    // runs of shared prefixes at least four candidates long on average
    struct Clustered {
        fem_ctx *c;
        bool saved;
        ~Clustered() { c->clustered = saved; }
    } restore{c, c->clustered};
    c->clustered = (uint64_t)m >= 4ull * ((uint64_t)info[2] + 1);
    if (info[1] && info[1] < m) {
        // distinct-type and repeated-type episodes mixed: count each part on its own
        // (repeated types run with one segment), then put the counts back in place
        uint8_t *rf;
        uint32_t *ridx, *rg, *rout, *scratch;
        RET(dbuf(c, "rep_flags", m, &rf));
        RET(dbuf(c, "rep_idx", m, &ridx));
        RET(dbuf(c, "rep_gather", m, &rg));
        RET(dbuf(c, "rep_out", m, &rout));
        RET(dbuf(c, "rep_scratch", compact_scratch_words(m), &scratch));
        for (bool rep : {false, true}) {
            CK(launch_repeat_flags(cands, gather, m, !rep, rf, st));
            CK(launch_compact(nullptr, rf, 0, m, ridx, c->d_small + W_COUNT2, scratch, st));
            uint32_t k;
            RET(read_words(c, c->d_small + W_COUNT2, 1, &k, st));
            if (!k) continue;
            CK(launch_compose_idx(gather, ridx, k, rg, st));
            RET(count_any(c, s, cands, rg, k, d_ivl, nI, pass, rout, st));
            CK(launch_scatter_u32(rout, ridx, k, out, st));
        }
        return FEM_OK;
    }
    const bool distinct = info[1] == 0;
    if (__builtin_popcount(lens) == 1) {
        const int N = __builtin_ctz(lens);
        return count_pass(c, s, cands, gather, m, N, d_ivl, nI, pass, out, distinct, st, nullptr);
    }
    uint8_t *flags;
    uint32_t *idx, *g2, *tmp, *scratch;
    RET(dbuf(c, "len_flags", m, &flags));
    RET(dbuf(c, "len_idx", m, &idx));
    RET(dbuf(c, "len_gather", m, &g2));
    RET(dbuf(c, "len_out", m, &tmp));
    RET(dbuf(c, "len_scratch", compact_scratch_words(m), &scratch));
    for (int N = 1; N <= FEM_MAX_LEN; ++N) {
        if (!(lens & (1u << N))) continue;
        CK(launch_len_flags(cands, gather, m, (uint32_t)N, flags, st));
        CK(launch_compact(nullptr, flags, 0, m, idx, c->d_small + W_COUNT1, scratch, st));
        uint32_t k;
        RET(read_words(c, c->d_small + W_COUNT1, 1, &k, st));
        if (!k) continue;
        CK(launch_compose_idx(gather, idx, k, g2, st));
        RET(count_pass(c, s, cands, g2, k, N, d_ivl, nI, pass, tmp, distinct, st, nullptr));
        CK(launch_scatter_u32(tmp, idx, k, out, st));
    }
    return FEM_OK;
}

void free_stream_buffers(StreamDev &s) {
    cudaFree(s.t);
    cudaFree(s.type);
    cudaFree(s.bev);
    cudaFree(s.boff);
    cudaFree(s.cfirst);
    cudaFree(s.hist);
    s = StreamDev{};
}

// Buffers for a stream of up to ne events in nc chunks (offs per chunk), charged to
// the context's budget as one block.
int alloc_stream(fem_ctx *c, StreamDev &s, size_t ne, size_t nc) {
    StreamDev q;
    q.cap_events = ne, q.cap_chunks = nc, q.cap_offs = (uint32_t)(nc * s.offs);
    q.t = reinterpret_cast<uint32_t *>(1);  // stream_bytes of the capacities
    const size_t bytes = stream_bytes(q);
    RET(reserve(c, bytes));
    s.cap_events = ne, s.cap_chunks = nc, s.cap_offs = q.cap_offs;
    const bool ok = cudaMalloc(&s.t, ne * 4) == cudaSuccess && cudaMalloc(&s.type, ne) == cudaSuccess &&
                    cudaMalloc(&s.bev, nc * CHUNK * 8) == cudaSuccess &&
                    cudaMalloc(&s.boff, nc * s.offs * 2) == cudaSuccess &&
                    cudaMalloc(&s.cfirst, (nc + 1) * 4) == cudaSuccess &&
                    cudaMalloc(&s.hist, 256 * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_stream_buffers(s);
        return FEM_ENOMEM;
    }
    c->mem_used += bytes;
    return FEM_OK;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

}  // extern "C"

namespace fem {
int fem_ctx_device(const fem_ctx *c) { return c->device; }
int fem_ctx_sms(const fem_ctx *c) { return c->sm_count; }
}  // namespace fem

extern "C" {

uint64_t fem_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char *fem_strerror(int s) {
    switch (s) {
        case FEM_OK: return "ok";
        case FEM_EINVAL: return "invalid argument";
        case FEM_EUNSORTED: return "stream times are not non-decreasing";
        case FEM_ETYPE: return "event type out of range";
        case FEM_ERANGE: return "time span plus interval bound exceeds 32 bits";
        case FEM_ENOMEM: return "out of memory";
        case FEM_EADMIT: return "request not admitted";
        case FEM_ETIMEOUT: return "bounded device wait timed out";
        case FEM_ECUDA: return "CUDA runtime error";
        case FEM_EOVERFLOW: return "internal capacity exceeded";
        case FEM_ENOSTREAM: return "unknown stream id";
        case FEM_EIO: return "file could not be opened, read or written";
        default: return "unknown status";
    }
}

int fem_create(fem_ctx **out, int device, size_t mem_budget_bytes) {
    if (!out) return FEM_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return FEM_ECUDA;
    }
    fem_ctx *c = new (std::nothrow) fem_ctx;
    if (!c) return FEM_ENOMEM;
    c->device = device;
    c->mem_budget = mem_budget_bytes;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&c->d_err, sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&c->d_small, 64 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&c->h_small, 64 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&c->h_load, (kLoadSeq + 1) * sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&c->h_ivl, (FEM_MAX_INTERVALS + 1) * sizeof(fem_interval)) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ivl_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&c->tev[0]) != cudaSuccess ||
        cudaEventCreate(&c->tev[1]) != cudaSuccess) {
        cudaGetLastError();
        fem_destroy(c);
        return FEM_ECUDA;
    }
    for (auto &set : c->kev) {
        for (auto &e : set) {
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                fem_destroy(c);
                return FEM_ECUDA;
            }
        }
    }
    for (auto &e : c->ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            fem_destroy(c);
            return FEM_ECUDA;
        }
    }
    cudaMemset(c->d_err, 0, sizeof(uint32_t));
    std::memset(c->h_small, 0, 64 * sizeof(uint32_t));  // no stale sequence number
    std::memset(c->h_load, 0, (kLoadSeq + 1) * sizeof(uint32_t));
    {
        void *dp = nullptr, *dl = nullptr;
        if (cudaHostGetDevicePointer(&dp, c->h_small, 0) == cudaSuccess && dp &&
            cudaHostGetDevicePointer(&dl, c->h_load, 0) == cudaSuccess && dl) {
            c->d_pub = static_cast<uint32_t *>(dp) + kPubWord;
            c->d_load = static_cast<uint32_t *>(dl);
        }
        cudaGetLastError();
    }
    *out = c;
    return FEM_OK;
}

int fem_destroy(fem_ctx *c) {
    if (!c) return FEM_EINVAL;
    cudaSetDevice(c->device);
    if (c->own) cudaStreamSynchronize(c->own);
    for (auto &kv : c->streams) free_stream_buffers(kv.second);
    for (auto &kv : c->bufs) cudaFree(kv.second.p);
    if (c->d_err) cudaFree(c->d_err);
    if (c->d_small) cudaFree(c->d_small);
    if (c->h_small) cudaFreeHost(c->h_small);
    if (c->h_load) cudaFreeHost(c->h_load);
    if (c->h_ivl) cudaFreeHost(c->h_ivl);
    if (c->ivl_ev) cudaEventDestroy(c->ivl_ev);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    for (auto &set : c->kev)
        for (auto &e : set)
            if (e) cudaEventDestroy(e);
    for (auto &e : c->tev)
        if (e) cudaEventDestroy(e);
    for (StreamDev &s : c->pool) free_stream_buffers(s);
    for (auto &b : c->pin)
        if (b.p) cudaFreeHost(b.p);
    if (c->own) cudaStreamDestroy(c->own);
    delete c;
    return FEM_OK;
}

int fem_set_config(fem_ctx *c, const fem_config *cfg) {
    if (!c) return FEM_EINVAL;
    if (!cfg) {
        c->cfg = fem_config{};
        return FEM_OK;
    }
    if (cfg->threads_per_block &&
        (cfg->threads_per_block % 32 || cfg->threads_per_block > 256))
        return FEM_EINVAL;
    if (cfg->ring_capacity && !count_config_supported(2, FEM_PASS_EXACT, false, cfg->ring_capacity))
        return FEM_EINVAL;
    if (cfg->kernel > FEM_KERNEL_CHAIN) return FEM_EINVAL;
    c->cfg = *cfg;
    return FEM_OK;
}

int fem_tune_enable(fem_ctx *c, int on) {
    if (!c) return FEM_EINVAL;
    c->tune_on = on != 0;
    return FEM_OK;
}

int fem_tune_size(fem_ctx *c, uint32_t *n_out) {
    if (!c || !n_out) return FEM_EINVAL;
    *n_out = (uint32_t)c->tune.size();
    return FEM_OK;
}

// One JSON object per line: {"key": "N/pass/distinct/log2m/log2chunks/K", "segments": P,
// "threads": T, "ms": t}
int fem_tune_save(fem_ctx *c, const char *path) {
    if (!c || !path) return FEM_EINVAL;
    FILE *f = std::fopen(path, "w");
    if (!f) return FEM_EIO;
    for (const auto &kv : c->tune)
        std::fprintf(f,
                     "{\"key\": \"%s\", \"segments\": %u, \"threads\": %u, \"ms\": %.6f, "
                     "\"kernel\": %u}\n",
                     kv.first.c_str(), kv.second.P, kv.second.T, kv.second.ms, kv.second.kernel);
    const bool ok = std::fclose(f) == 0;
    return ok ? FEM_OK : FEM_EIO;
}

int fem_tune_load(fem_ctx *c, const char *path) {
    if (!c || !path) return FEM_EINVAL;
    FILE *f = std::fopen(path, "r");
    if (!f) return FEM_EIO;
    std::map<std::string, fem_ctx::Shape> got;
    char line[512];
    int rc = FEM_OK;
    while (std::fgets(line, sizeof(line), f)) {
        if (line[0] == '\n' || line[0] == 0) continue;
        char key[96];
        unsigned P = 0, T = 0, K = FEM_KERNEL_MACHINE;
        float ms = 0;
        char close = 0;
        const int nf = std::sscanf(
            line, " {\"key\": \"%95[0-9/]\", \"segments\": %u, \"threads\": %u, \"ms\": %f%c",
            key, &P, &T, &ms, &close);
        bool good = nf == 5 && P != 0 && T != 0 && T <= 256 && T % 8 == 0;
        if (good && close == ',') {  // with the kernel field
            good = std::sscanf(std::strstr(line, "\"ms\""), "\"ms\": %*f, \"kernel\": %u}", &K) == 1 &&
                   (K == FEM_KERNEL_MACHINE || K == FEM_KERNEL_CHAIN);
        } else if (good) {
            good = close == '}';
        }
        if (!good) {
            rc = FEM_EINVAL;
            break;
        }
        got[key] = fem_ctx::Shape{P, T, ms, K};
    }
    std::fclose(f);
    if (rc != FEM_OK) return rc;
    for (auto &kv : got) c->tune[kv.first] = kv.second;
    return FEM_OK;
}

int fem_load_stream(fem_ctx *c, const uint8_t *types, const uint32_t *t_us, uint64_t n,
                    uint32_t n_types, int on_device, void *cuda_stream, int32_t *id_out) {
    if (!c || !id_out || n_types == 0 || n_types > FEM_MAX_TYPES) return FEM_EINVAL;
    if (n && (!types || !t_us)) return FEM_EINVAL;
    if (n >= 0xFFFFFFF0ull) return FEM_EINVAL;
    cudaSetDevice(c->device);
    cudaStream_t st = pick(c, cuda_stream);
    StreamDev s;
    s.n = n;
    s.K = n_types;
    s.n_chunks = (uint32_t)((n + CHUNK - 1) / CHUNK);
    s.offs = offs_stride(n_types);
    const size_t nn = std::max<uint64_t>(n, 1);
    const size_t nc = std::max<uint32_t>(s.n_chunks, 1);
    bool okm = false;
    for (size_t i = 0; i < c->pool.size(); ++i) {
        StreamDev &q = c->pool[i];
        if (q.cap_events >= nn && q.cap_chunks >= nc && q.cap_offs >= nc * s.offs) {
            s.t = q.t, s.type = q.type, s.bev = q.bev, s.boff = q.boff, s.cfirst = q.cfirst,
            s.hist = q.hist;
            s.cap_events = q.cap_events, s.cap_chunks = q.cap_chunks, s.cap_offs = q.cap_offs;
            c->pool.erase(c->pool.begin() + i);
            okm = true;
            break;
        }
    }
    if (!okm) okm = alloc_stream(c, s, nn, nc) == FEM_OK;
    auto release = [&] {
        c->mem_used -= std::min(stream_bytes(s), c->mem_used);
        free_stream_buffers(s);
    };
    if (!okm) return FEM_ENOMEM;
    int rc = FEM_OK;
    std::vector<uint32_t> hist_host;
    do {
        // the histogram is cleared here (k_bucket accumulates into it); the chunk start
        // times are all written by k_bucket, and need filling only for an empty stream
        if (cudaMemsetAsync(c->d_err, 0, 4, st) != cudaSuccess ||
            cudaMemsetAsync(s.hist, 0, 256 * 4, st) != cudaSuccess ||
            (!n && cudaMemsetAsync(s.cfirst, 0xFF, (nc + 1) * 4, st) != cudaSuccess)) {
            rc = FEM_ECUDA;
            break;
        }
        if (n && on_device) {  // one kernel reads, checks, copies and groups the events
            if (launch_load_stream(s, st, c->d_err, t_us, types) != cudaSuccess) {
                rc = FEM_ECUDA;
                break;
            }
        } else if (n) {
            if (cudaMemcpyAsync(s.t, t_us, n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(s.type, types, n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                launch_load_stream(s, st, c->d_err) != cudaSuccess) {
                rc = FEM_ECUDA;
                break;
            }
        }
        // error word, last time and type histogram in one round trip: published by a
        // kernel into mapped words, else copied
        if (c->d_load) {
            const uint32_t seq = ++c->pub_seq;
            if (launch_publish_load(c->d_err, n ? s.t + (n - 1) : nullptr, s.hist, n_types,
                                    c->d_load, kLoadSeq, seq, st) != cudaSuccess) {
                rc = FEM_ECUDA;
                break;
            }
            if ((rc = wait_seq(c->h_load + kLoadSeq, seq, st)) != FEM_OK) break;
            const volatile uint32_t *hv = c->h_load;
            if ((rc = err_status(hv[0])) != FEM_OK) break;
            if (n) s.t_max = hv[1];
            hist_host.assign(n_types, 0);
            for (uint32_t a = 0; a < n_types; ++a) hist_host[a] = hv[2 + a];
            break;
        }
        void *hp;
        if ((rc = pinbuf(c, 0, (2 + 256) * sizeof(uint32_t), st, &hp)) != FEM_OK) break;
        uint32_t *hw = static_cast<uint32_t *>(hp);
        if (cudaMemcpyAsync(hw, c->d_err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            (n && cudaMemcpyAsync(hw + 1, s.t + (n - 1), 4, cudaMemcpyDeviceToHost, st) !=
                      cudaSuccess) ||
            cudaMemcpyAsync(hw + 2, s.hist, n_types * 4, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = FEM_ECUDA;
            break;
        }
        if ((rc = err_status(hw[0])) != FEM_OK) break;
        if (n) s.t_max = hw[1];
        hist_host.assign(hw + 2, hw + 2 + n_types);
    } while (0);
    if (rc != FEM_OK) {
        cudaGetLastError();
        cudaStreamSynchronize(st);
        release();
        return rc;
    }
    const int32_t id = c->next_id++;
    s.gen = c->next_gen++;
    c->streams[id] = s;
    c->hist_h[id] = std::move(hist_host);
    *id_out = id;
    return FEM_OK;
}

int fem_append_stream(fem_ctx *c, int32_t id, const uint8_t *types, const uint32_t *t_us,
                      uint64_t n, int on_device, void *cuda_stream) {
    if (!c || (n && (!types || !t_us))) return FEM_EINVAL;
    auto it = c->streams.find(id);
    if (it == c->streams.end()) return FEM_ENOSTREAM;
    if (n == 0) return FEM_OK;
    StreamDev &s = it->second;
    const uint64_t n_old = s.n, n_new = s.n + n;
    if (n_new >= 0xFFFFFFF0ull) return FEM_EINVAL;
    cudaSetDevice(c->device);
    cudaStream_t st = pick(c, cuda_stream);
    const uint32_t ch_old = s.n_chunks, K = s.K, t_max_old = s.t_max;
    const uint32_t ch_new = (uint32_t)((n_new + CHUNK - 1) / CHUNK);
    if (n_new > s.cap_events || ch_new > s.cap_chunks || (uint64_t)ch_new * s.offs > s.cap_offs) {
        // grow by half at least, keeping what is grouped already
        StreamDev g;
        g.offs = s.offs;
        RET(alloc_stream(c, g, std::max<uint64_t>(n_new, s.cap_events * 3 / 2),
                         std::max<uint64_t>(ch_new, s.cap_chunks * 3 / 2)));
        bool ok = true;
        if (n_old) {
            ok = cudaMemcpyAsync(g.t, s.t, n_old * 4, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
                 cudaMemcpyAsync(g.type, s.type, n_old, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
                 cudaMemcpyAsync(g.bev, s.bev, (size_t)ch_old * CHUNK * 8, cudaMemcpyDeviceToDevice,
                                 st) == cudaSuccess &&
                 cudaMemcpyAsync(g.boff, s.boff, (size_t)ch_old * s.offs * 2,
                                 cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
                 cudaMemcpyAsync(g.cfirst, s.cfirst, ((size_t)ch_old + 1) * 4,
                                 cudaMemcpyDeviceToDevice, st) == cudaSuccess;
        }
        ok = ok && cudaMemcpyAsync(g.hist, s.hist, 256 * 4, cudaMemcpyDeviceToDevice, st) ==
                       cudaSuccess &&
             cudaStreamSynchronize(st) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            c->mem_used -= std::min(stream_bytes(g), c->mem_used);
            free_stream_buffers(g);
            return FEM_ECUDA;
        }
        c->mem_used -= std::min(stream_bytes(s), c->mem_used);
        free_stream_buffers(s);
        g.n = n_old, g.K = K, g.n_chunks = ch_old, g.t_max = t_max_old;
        s = g;
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemsetAsync(c->d_err, 0, 4, st));
    CK(cudaMemcpyAsync(s.t + n_old, t_us, n * 4, kind, st));
    CK(cudaMemcpyAsync(s.type + n_old, types, n, kind, st));
    s.n = n_new;
    s.n_chunks = ch_new;
    // regroup from the chunk holding the old last event, so that the pair across the old
    // end is checked with the new events
    const uint32_t c0 = n_old ? (uint32_t)((n_old - 1) / CHUNK) : 0u;
    CK(launch_bucket_chunks(s, c0, ch_new, st, c->d_err));
    CK(launch_hist_add(s.type + n_old, n, s.K, +1, s.hist, st));
    void *hp;
    RET(pinbuf(c, 0, (2 + 256) * sizeof(uint32_t), st, &hp));
    uint32_t *hw = static_cast<uint32_t *>(hp);
    CK(cudaMemcpyAsync(hw, c->d_err, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hw + 1, s.t + (n_new - 1), 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hw + 2, s.hist, s.K * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int rc = err_status(hw[0]);
    if (rc != FEM_OK) {
        // undo: the old events' grouping, histogram and size
        CK(launch_hist_add(s.type + n_old, n, s.K, -1, s.hist, st));
        s.n = n_old;
        s.n_chunks = ch_old;
        if (n_old) CK(launch_bucket_chunks(s, c0, ch_old, st));
        else CK(cudaMemsetAsync(s.cfirst, 0xFF, 8, st));
        CK(cudaStreamSynchronize(st));
        s.t_max = t_max_old;
        return rc;
    }
    s.t_max = hw[1];
    s.gen = c->next_gen++;
    c->hist_h[id].assign(hw + 2, hw + 2 + s.K);
    return FEM_OK;
}

int fem_mem_usage(fem_ctx *c, size_t *used_out, size_t *budget_out) {
    if (!c) return FEM_EINVAL;
    if (used_out) *used_out = c->mem_used;
    if (budget_out) *budget_out = c->mem_budget;
    return FEM_OK;
}

int fem_free_stream(fem_ctx *c, int32_t id) {
    if (!c) return FEM_EINVAL;
    auto it = c->streams.find(id);
    if (it == c->streams.end()) return FEM_ENOSTREAM;
    cudaSetDevice(c->device);
    // Keep the buffers for the next load (work already queued that reads them runs
    // first: every stream of this context is synchronised before reuse).
    cudaDeviceSynchronize();
    c->pool.push_back(it->second);
    c->streams.erase(it);
    c->hist_h.erase(id);
    while (c->pool.size() > 4) {
        c->mem_used -= std::min(stream_bytes(c->pool.front()), c->mem_used);
        free_stream_buffers(c->pool.front());
        c->pool.erase(c->pool.begin());
    }
    return FEM_OK;
}

int fem_type_counts(fem_ctx *c, int32_t id, uint32_t *counts_out) {
    if (!c || !counts_out) return FEM_EINVAL;
    const StreamDev *s = find_stream(c, id);
    if (!s) return FEM_ENOSTREAM;
    cudaSetDevice(c->device);
    CK(cudaMemcpyAsync(counts_out, s->hist, s->K * 4, cudaMemcpyDeviceToHost, c->own));
    CK(cudaStreamSynchronize(c->own));
    return FEM_OK;
}

int fem_capacity_table(fem_ctx *c, int32_t id, const uint32_t *widths, uint32_t nh,
                       uint32_t *cap_out) {
    if (!c || !widths || !cap_out || nh == 0 || nh > FEM_MAX_CAP_WIDTHS) return FEM_EINVAL;
    const StreamDev *s = find_stream(c, id);
    if (!s) return FEM_ENOSTREAM;
    cudaSetDevice(c->device);
    return capacity(c, *s, widths, nh, cap_out, c->own);
}

int fem_count_pairs_relaxed(fem_ctx *c, int32_t id, const uint8_t *types, uint32_t f,
                            const fem_interval *I, uint32_t nI, uint32_t *counts_out) {
    if (!c || !types || !counts_out || f < 2 || f > 256 || nI == 0 || nI > 4) return FEM_EINVAL;
    const StreamDev *s = find_stream(c, id);
    if (!s) return FEM_ENOSTREAM;
    RET(check_intervals(*s, I, nI));
    bool seen[256] = {};
    for (uint32_t i = 0; i < f; ++i) {
        if (types[i] >= s->K || seen[types[i]]) return FEM_EINVAL;
        seen[types[i]] = true;
    }
    cudaSetDevice(c->device);
    cudaStream_t st = c->own;
    CK(cudaMemsetAsync(c->d_err, 0, 4, st));
    uint2 *d_ivl;
    RET(upload_intervals(c, I, nI, st, &d_ivl));
    const uint32_t m = f * (f - 1) * nI;
    uint32_t *ft, *out;
    fem_episode *cands;
    RET(dbuf(c, "pair_types", f, &ft));
    RET(dbuf(c, "pair_cands", m, &cands));
    RET(dbuf(c, "pair_out", m, &out));
    std::vector<uint32_t> ftv(types, types + f);
    CK(cudaMemcpyAsync(ft, ftv.data(), f * 4, cudaMemcpyHostToDevice, st));
    CK(launch_level2(ft, f, nI, false, cands, st));
    PassLaunch pl;
    RET(count_launch_pairs(c, *s, cands, m, f, d_ivl, nI, out, st, &pl));
    uint32_t e;
    RET(read_err(c, st, &e));
    RET(count_finish(c, *s, pl, e, st));
    CK(cudaMemcpyAsync(counts_out, out, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return FEM_OK;
}

int fem_count_candidates(fem_ctx *c, int32_t id, const fem_episode *cands, uint32_t m,
                         int cands_on_device, const fem_interval *I, uint32_t nI, int pass,
                         uint32_t *counts_out, int counts_on_device, void *cuda_stream) {
    if (!c || (m && (!cands || !counts_out))) return FEM_EINVAL;
    if (pass != FEM_PASS_RELAXED && pass != FEM_PASS_EXACT) return FEM_EINVAL;
    const StreamDev *s = find_stream(c, id);
    if (!s) return FEM_ENOSTREAM;
    RET(check_intervals(*s, I, nI));
    if (m == 0) return FEM_OK;
    cudaSetDevice(c->device);
    cudaStream_t st = pick(c, cuda_stream);
    CK(cudaMemsetAsync(c->d_err, 0, 4, st));
    uint2 *d_ivl;
    RET(upload_intervals(c, I, nI, st, &d_ivl));
    const fem_episode *dc = cands;
    if (!cands_on_device) {
        fem_episode *tmp;
        RET(dbuf(c, "cands_in", m, &tmp));
        CK(cudaMemcpyAsync(tmp, cands, (size_t)m * sizeof(fem_episode), cudaMemcpyHostToDevice, st));
        dc = tmp;
    }
    uint32_t *dout = counts_out;
    if (!counts_on_device) RET(dbuf(c, "counts_out", m, &dout));
    RET(count_any(c, *s, dc, nullptr, m, d_ivl, nI, pass, dout, st));
    if (!counts_on_device) {
        CK(cudaMemcpyAsync(counts_out, dout, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return FEM_OK;
}

int fem_count_mapconcat_literal(fem_ctx *c, int32_t id, const fem_episode *cands, uint32_t m,
                                int cands_on_device, const fem_interval *I, uint32_t nI,
                                uint32_t segments, uint32_t *counts_out, int counts_on_device,
                                uint32_t *diag_out, void *cuda_stream) {
    if (!c || (m && (!cands || !counts_out))) return FEM_EINVAL;
    const StreamDev *s = find_stream(c, id);
    if (!s) return FEM_ENOSTREAM;
    RET(check_intervals(*s, I, nI));
    if (diag_out) diag_out[0] = diag_out[1] = 0;
    if (m == 0) return FEM_OK;
    cudaSetDevice(c->device);
    cudaStream_t st = pick(c, cuda_stream);
    CK(cudaMemsetAsync(c->d_err, 0, 4, st));
    uint2 *d_ivl;
    RET(upload_intervals(c, I, nI, st, &d_ivl));
    const fem_episode *dc = cands;
    if (!cands_on_device) {
        fem_episode *tmp;
        RET(dbuf(c, "cands_in", m, &tmp));
        CK(cudaMemcpyAsync(tmp, cands, (size_t)m * sizeof(fem_episode), cudaMemcpyHostToDevice, st));
        dc = tmp;
    }
    uint32_t *dout = counts_out;
    if (!counts_on_device) RET(dbuf(c, "counts_out", m, &dout));
    // the printed scheme needs distinct types (as the exact MapConcatenate does)
    CK(cudaMemsetAsync(c->d_small + W_INFO, 0, 3 * sizeof(uint32_t), st));
    CK(launch_validate_cands(dc, nullptr, m, s->K, nI, c->d_small + W_INFO, c->d_err, st));
    uint32_t info[3], e;
    RET(read_words(c, c->d_small + W_INFO, 3, info, st));
    RET(read_err(c, st, &e));
    RET(err_status(e));
    if (info[1]) return FEM_EINVAL;
    if (s->n == 0) {
        CK(cudaMemsetAsync(dout, 0, (size_t)m * 4, st));
    } else {
        // time cuts at the first event of every cps-th chunk (dropped where equal
        // times would make them non-increasing)
        std::vector<uint32_t> cf(s->n_chunks + 1);
        CK(cudaMemcpyAsync(cf.data(), s->cfirst, cf.size() * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const uint32_t P0 = std::max<uint32_t>(1, std::min<uint32_t>(segments ? segments : 1,
                                                                     s->n_chunks));
        const uint32_t cps = (s->n_chunks + P0 - 1) / P0;
        std::vector<int64_t> tau{(int64_t)cf[0] - 1};
        for (uint32_t c0 = cps; c0 < s->n_chunks; c0 += cps)
            if ((int64_t)cf[c0] - 1 > tau.back() && (int64_t)cf[c0] - 1 < (int64_t)s->t_max)
                tau.push_back((int64_t)cf[c0] - 1);
        tau.push_back((int64_t)s->t_max);
        const uint32_t P = (uint32_t)tau.size() - 1;
        int64_t *d_tau;
        uint4 *tuples;
        RET(dbuf(c, "lit_tau", tau.size(), &d_tau));
        RET(dbuf(c, "lit_tuples", (size_t)m * P * FEM_MAX_LEN, &tuples));
        CK(cudaMemcpyAsync(d_tau, tau.data(), tau.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                           st));
        CK(cudaMemsetAsync(c->d_small + W_INFO, 0, 2 * sizeof(uint32_t), st));
        LiteralParams p{};
        p.bev = s->bev;
        p.boff = s->boff;
        p.t = s->t;
        p.offs = s->offs;
        p.n = s->n;
        p.cands = dc;
        p.m = m;
        p.ivl = d_ivl;
        p.tau = d_tau;
        p.P = P;
        p.tuples = tuples;
        p.err = c->d_err;
        CK(launch_literal(p, info[0], dout, c->d_small + W_INFO, st));
        uint32_t dg[2];
        RET(read_words(c, c->d_small + W_INFO, 2, dg, st));
        RET(read_err(c, st, &e));
        if (e & ERR_RING) return FEM_EOVERFLOW;
        RET(err_status(e));
        if (diag_out) diag_out[0] = dg[0], diag_out[1] = dg[1];
    }
    if (!counts_on_device) {
        CK(cudaMemcpyAsync(counts_out, dout, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return FEM_OK;
}

int fem_count_windows(fem_ctx *c, int32_t id, const fem_episode *cands, uint32_t m,
                      int cands_on_device, const fem_interval *I, uint32_t nI, uint32_t window_us,
                      uint64_t *counts_out, int counts_on_device, void *cuda_stream) {
    if (!c || (m && (!cands || !counts_out)) || window_us == 0) return FEM_EINVAL;
    const StreamDev *s = find_stream(c, id);
    if (!s) return FEM_ENOSTREAM;
    RET(check_intervals(*s, I, nI));
    if (m == 0) return FEM_OK;
    cudaSetDevice(c->device);
    cudaStream_t st = pick(c, cuda_stream);
    CK(cudaMemsetAsync(c->d_err, 0, 4, st));
    uint2 *d_ivl;
    RET(upload_intervals(c, I, nI, st, &d_ivl));
    const fem_episode *dc = cands;
    if (!cands_on_device) {
        fem_episode *tmp;
        RET(dbuf(c, "cands_in", m, &tmp));
        CK(cudaMemcpyAsync(tmp, cands, (size_t)m * sizeof(fem_episode), cudaMemcpyHostToDevice, st));
        dc = tmp;
    }
    uint64_t *dout = counts_out;
    if (!counts_on_device) RET(dbuf(c, "win_out", m, &dout));
    CK(cudaMemsetAsync(c->d_small + W_INFO, 0, 3 * sizeof(uint32_t), st));
    CK(launch_validate_cands(dc, nullptr, m, s->K, nI, c->d_small + W_INFO, c->d_err, st));
    uint32_t info[3], e;
    RET(read_words(c, c->d_small + W_INFO, 3, info, st));
    RET(read_err(c, st, &e));
    RET(err_status(e));
    if (info[1]) return FEM_EINVAL;  // distinct types only
    WindowParams p{};
    p.bev = s->bev;
    p.boff = s->boff;
    p.offs = s->offs;
    p.n = s->n;
    p.cands = dc;
    p.m = m;
    p.ivl = d_ivl;
    p.w = window_us;
    p.out = dout;
    p.err = c->d_err;
    CK(launch_count_windows(p, info[0], st));
    RET(read_err(c, st, &e));
    if (e & ERR_RING) return FEM_EOVERFLOW;
    RET(err_status(e));
    if (!counts_on_device) {
        CK(cudaMemcpyAsync(counts_out, dout, (size_t)m * 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return FEM_OK;
}

int fem_count_two_pass(fem_ctx *c, int32_t id, const fem_episode *cands, uint32_t m,
                       int cands_on_device, const fem_interval *I, uint32_t nI, uint32_t theta,
                       uint32_t *exact_out, uint8_t *survived_out, int outs_on_device,
                       void *cuda_stream) {
    if (!c || (m && !cands)) return FEM_EINVAL;
    const StreamDev *s = find_stream(c, id);
    if (!s) return FEM_ENOSTREAM;
    RET(check_intervals(*s, I, nI));
    if (m == 0) return FEM_OK;
    cudaSetDevice(c->device);
    cudaStream_t st = pick(c, cuda_stream);
    CK(cudaMemsetAsync(c->d_err, 0, 4, st));
    uint2 *d_ivl;
    RET(upload_intervals(c, I, nI, st, &d_ivl));
    const fem_episode *dc = cands;
    if (!cands_on_device) {
        fem_episode *tmp;
        RET(dbuf(c, "cands_in", m, &tmp));
        CK(cudaMemcpyAsync(tmp, cands, (size_t)m * sizeof(fem_episode), cudaMemcpyHostToDevice, st));
        dc = tmp;
    }
    uint32_t *rel, *idx, *ex, *exo, *scratch;
    uint8_t *sv;
    RET(dbuf(c, "tp_rel", m, &rel));
    RET(dbuf(c, "tp_idx", m, &idx));
    RET(dbuf(c, "tp_ex", m, &ex));
    RET(dbuf(c, "scratch", compact_scratch_words(m), &scratch));
    exo = (outs_on_device && exact_out) ? exact_out : nullptr;
    if (!exo) RET(dbuf(c, "tp_exo", m, &exo));
    sv = (outs_on_device && survived_out) ? survived_out : nullptr;
    if (!sv) RET(dbuf(c, "tp_sv", m, &sv));
    // first pass: relaxed counts, eliminate count < theta
    RET(count_any(c, *s, dc, nullptr, m, d_ivl, nI, FEM_PASS_RELAXED, rel, st));
    CK(launch_compact(rel, nullptr, theta, m, idx, c->d_small + W_COUNT0, scratch, st, pub_of(c)));
    uint32_t ms, e0;
    RET(read_count_err(c, c->d_small + W_COUNT0, &ms, &e0, st));
    RET(err_status(e0));
    // second pass: exact counts of the survivors
    RET(count_any(c, *s, dc, idx, ms, d_ivl, nI, FEM_PASS_EXACT, ex, st));
    CK(cudaMemsetAsync(exo, 0, (size_t)m * 4, st));
    CK(cudaMemsetAsync(sv, 0, m, st));
    CK(launch_scatter_u32(ex, idx, ms, exo, st));
    CK(launch_fill_flags(idx, ms, sv, st));
    if (!outs_on_device) {
        if (exact_out) CK(cudaMemcpyAsync(exact_out, exo, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
        if (survived_out) CK(cudaMemcpyAsync(survived_out, sv, m, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    return FEM_OK;
}

int fem_mine_levelwise(fem_ctx *c, int32_t id, const fem_interval *I, uint32_t nI,
                       uint32_t theta, uint32_t max_len, void *cuda_stream, fem_result **out) {
    return fem_mine_levelwise_ex(c, id, I, nI, theta, max_len, 0u, cuda_stream, out);
}

int fem_mine_levelwise_ex(fem_ctx *c, int32_t id, const fem_interval *I, uint32_t nI,
                          uint32_t theta, uint32_t max_len, uint32_t flags, void *cuda_stream,
                          fem_result **out) {
    if (!c || !out || max_len < 1 || max_len > FEM_MAX_LEN) return FEM_EINVAL;
    if (flags & ~FEM_MINE_REPEATED_TYPES) return FEM_EINVAL;
    const bool repeats = (flags & FEM_MINE_REPEATED_TYPES) != 0;
    *out = nullptr;
    const StreamDev *sp = find_stream(c, id);
    if (!sp) return FEM_ENOSTREAM;
    const StreamDev &s = *sp;
    RET(check_intervals(s, I, nI));
    cudaSetDevice(c->device);
    cudaStream_t st = pick(c, cuda_stream);
    CK(cudaMemsetAsync(c->d_err, 0, 4, st));
    c->stats.clear();
    fem_result *res = new (std::nothrow) fem_result;
    if (!res) return FEM_ENOMEM;
    res->eps.resize(max_len);
    res->counts.resize(max_len);
    auto fail = [&](int rc) {
        delete res;
        return rc;
    };
#define RETF(x)                         \
    do {                                \
        int r_ = (x);                   \
        if (r_ != FEM_OK) return fail(r_); \
    } while (0)
#define CKF(x)                                         \
    do {                                               \
        if ((x) != cudaSuccess) return fail(FEM_ECUDA); \
    } while (0)

    uint2 *d_ivl;
    RETF(upload_intervals(c, I, nI, st, &d_ivl));
    // per level, the (episode, event) pairs each pass visits (statistics only)
    unsigned long long *touched;
    RETF(dbuf(c, "touched", 2 * (FEM_MAX_LEN + 1), &touched));
    CKF(cudaMemsetAsync(touched, 0, 2 * (FEM_MAX_LEN + 1) * sizeof(unsigned long long), st));
    // level 1: the count of a one-node episode is the number of events of its type.
    // The device keeps the frequent types for generating level 2; the host takes the
    // same types (the same comparison) from the histogram the load read back, so it
    // needs no round trip to size level 2.
    uint32_t *ftypes;
    RETF(dbuf(c, "ftypes", 256, &ftypes));
    CKF(launch_type_filter(s.hist, s.K, theta, ftypes, c->d_small + W_COUNT0, st));
    const std::vector<uint32_t> &hist = c->hist_h[id];
    if (hist.size() != s.K) return fail(FEM_EINVAL);
    uint32_t f1 = 0;
    for (uint32_t a = 0; a < s.K; ++a) {
        if (!(hist[a] >= theta)) continue;
        fem_episode e;
        std::memset(&e, 0, sizeof(e));
        e.types[0] = (uint8_t)a;
        e.len = 1;
        res->eps[0].push_back(e);
        res->counts[0].push_back(hist[a]);
        ++f1;
    }
    if (max_len < 2 || f1 < (repeats ? 1u : 2u) || nI == 0) {
        *out = res;
        return FEM_OK;
    }
    uint64_t m64 = (uint64_t)f1 * nI * (repeats ? f1 : f1 - 1);
    if (m64 > 0xFFFFFFF0ull) return fail(FEM_ENOMEM);
    uint32_t m = (uint32_t)m64;
    // level 2: ordered pairs of distinct frequent types x intervals.  Its relaxed pass
    // runs on the pair kernel (fem_pairs.cu) unless a kernel is configured or a shape
    // was measured or loaded for the pass's class: with two or more intervals a thread
    // shares one merge of a pair's events among its variants (on the 64-type
    // recording 0.26 ms against 0.29 for one thread per candidate)
    const bool pairs_level2 =
        !repeats && !c->cfg.kernel && nI >= 2 && nI <= 4 &&
        c->tune.find(tune_key(2, FEM_PASS_RELAXED, true, m, s.n_chunks, s.K)) == c->tune.end();
    const char *cname[2] = {"candsA", "candsB"};
    int cur = 0;
    fem_episode *cands;
    RETF(dbuf(c, cname[cur], m, &cands));
    cudaEventRecord(c->ev[0], st);
    CKF(launch_level2(ftypes, f1, nI, repeats, cands, st));
    cudaEventRecord(c->ev[1], st);
    // Per level the host waits three times: for the survivor count, the frequent
    // count and the next level's candidate count (each read together with the error
    // word; capacity recounts, when flagged, run before the count is used).
    // Timings are read from events after those waits; frequent sets are copied to
    // pinned staging and moved into the result after the last wait.
    uint32_t staged_f[FEM_MAX_LEN + 1] = {};
    auto compact_and_read = [&](const uint32_t *vals, uint32_t mm, uint32_t *idx, uint32_t word,
                                uint32_t *scratch, const PassLaunch &pl, uint32_t *kept,
                                cudaEvent_t done) -> int {
        CK(launch_compact(vals, nullptr, theta, mm, idx, c->d_small + word, scratch, st, pub_of(c)));
        if (done) CK(cudaEventRecord(done, st));
        uint32_t e;
        RET(read_count_err(c, c->d_small + word, kept, &e, st));
        if (e & ERR_CAP) {
            RET(count_finish(c, s, pl, e, st));
            CK(launch_compact(vals, nullptr, theta, mm, idx, c->d_small + word, scratch, st,
                              pub_of(c)));
            RET(read_count_err(c, c->d_small + word, kept, &e, st));
        }
        return err_status(e);
    };
    for (uint32_t N = 2; N <= max_len && m > 0; ++N) {
        fem_level_stats ls{};
        ls.level = N;
        ls.candidates = m;
        uint32_t *rel, *idx_s, *ex, *idx_f, *fcnt, *scratch;
        fem_episode *F;
        RETF(dbuf(c, "rel", m, &rel));
        RETF(dbuf(c, "idx_s", m, &idx_s));
        RETF(dbuf(c, "scratch", compact_scratch_words(m), &scratch));
        // first pass (Algorithm 3) on every candidate, then eliminate relaxed < theta
        PassLaunch plr;
        cudaEventRecord(c->ev[2], st);
        if (repeats) {  // repeated types among the candidates: split and count (count_any)
            RETF(count_any(c, s, cands, nullptr, m, d_ivl, nI, FEM_PASS_RELAXED, rel, st));
        } else if (N == 2 && pairs_level2) {
            // every interval variant of an ordered type pair from one merge; the
            // candidates it gives up on go to the exact pass unfiltered when they are
            // at most 1/64 of the level, else to the recount
            uint32_t *work;
            RETF(dbuf(c, "pairs_work", 2, &work));
            CKF(cudaMemsetAsync(work, 0, 2 * sizeof(uint32_t), st));
            RETF(count_launch_pairs(c, s, cands, m, f1, d_ivl, nI, rel, st, &plr));
            CKF(launch_pairs_pass_flagged(rel, plr.p.redo, m, m / 64, work, c->d_err, st));
        } else {
            RETF(count_launch(c, s, cands, nullptr, m, (int)N, d_ivl, nI, FEM_PASS_RELAXED, rel,
                              true, st, &plr));
        }
        cudaEventRecord(c->ev[3], st);
        cudaEventRecord(c->ev[4], st);
        uint32_t ms;
        RETF(compact_and_read(rel, m, idx_s, W_COUNT0, scratch, plr, &ms, c->ev[5]));
        ls.survivors = ms;
        // second pass (Algorithm 1) on the survivors, then keep exact >= theta; the
        // relaxed pass's times are read and its statistics queued after this launch, so
        // that the device does not wait for the host's bookkeeping
        RETF(dbuf(c, "ex", ms, &ex));
        RETF(dbuf(c, "idx_f", ms, &idx_f));
        PassLaunch plx;
        cudaEventRecord(c->ev[6], st);
        if (repeats)
            RETF(count_any(c, s, cands, idx_s, ms, d_ivl, nI, FEM_PASS_EXACT, ex, st));
        else
            RETF(count_launch(c, s, cands, idx_s, ms, (int)N, d_ivl, nI, FEM_PASS_EXACT, ex, true,
                              st, &plx));
        cudaEventRecord(c->ev[7], st);
        PassInfo pi;
        pass_info(c, plr, &pi);
        cudaEventElapsedTime(&ls.ms_generate, c->ev[0], c->ev[1]);
        cudaEventElapsedTime(&ls.ms_relaxed, c->ev[2], c->ev[3]);
        ls.segments = pi.segments;
        ls.kernel_relaxed = pi.kernel;
        ls.ms_relaxed_kernel = pi.ms_kernel;
        ls.ms_relaxed_stitch = pi.ms_stitch;
        uint32_t f = 0;
        if (ms) RETF(compact_and_read(ex, ms, idx_f, W_COUNT1, scratch, plx, &f, nullptr));
        // work statistics of both passes (idx_s and the candidates stay until the next
        // level): queued behind the next wait's publishing launch where there is one
        auto queue_touched = [&]() -> int {
            CK(launch_touched(cands, nullptr, m, s.hist, touched + 2 * N, st));
            CK(launch_touched(cands, idx_s, ms, s.hist, touched + 2 * N + 1, st));
            return FEM_OK;
        };
        PassInfo pe;
        pass_info(c, plx, &pe);
        cudaEventElapsedTime(&ls.ms_compact, c->ev[4], c->ev[5]);
        cudaEventElapsedTime(&ls.ms_exact, c->ev[6], c->ev[7]);
        ls.ms_exact_kernel = pe.ms_kernel;
        ls.exact_segments = ms ? pe.segments : 0;
        ls.kernel_exact = ms ? pe.kernel : 0;
        ls.frequent = f;
        c->stats.push_back(ls);
        if (f == 0) {
            RETF(queue_touched());
            break;
        }
        RETF(dbuf(c, "fcnt", f, &fcnt));
        RETF(dbuf(c, "F", f, &F));
        CKF(launch_gather_frequent(cands, idx_s, idx_f, f, ex, F, fcnt, st));
        void *h;
        RETF(pinbuf(c, N, (size_t)f * (sizeof(fem_episode) + 4), st, &h));
        CKF(cudaMemcpyAsync(h, F, (size_t)f * sizeof(fem_episode), cudaMemcpyDeviceToHost, st));
        CKF(cudaMemcpyAsync(static_cast<uint8_t *>(h) + (size_t)f * sizeof(fem_episode), fcnt,
                            (size_t)f * 4, cudaMemcpyDeviceToHost, st));
        staged_f[N] = f;
        if (N == max_len) {
            RETF(queue_touched());
            break;
        }
        // join level N -> N + 1
        uint32_t *jc, *joff;
        RETF(dbuf(c, "jc", f, &jc));
        RETF(dbuf(c, "joff", f, &joff));
        cudaEventRecord(c->ev[0], st);
        CKF(launch_join_count(F, f, N, repeats, jc, c->sm_count, st));
        CKF(launch_exclusive_scan(jc, f, joff, c->d_small + W_COUNT2, scratch, st, pub_of(c)));
        RETF(queue_touched());
        uint32_t mn, ej;
        RETF(read_count_err(c, c->d_small + W_COUNT2, &mn, &ej, st));
        RETF(err_status(ej));
        cur ^= 1;
        RETF(dbuf(c, cname[cur], std::max<uint32_t>(mn, 1), &cands));
        CKF(launch_join_emit(F, f, N, repeats, joff, cands, c->sm_count, st));
        cudaEventRecord(c->ev[1], st);
        m = mn;
    }
    // statistics and the error word in the last round trip (pinned words)
    constexpr size_t TB = 2 * (FEM_MAX_LEN + 1) * sizeof(unsigned long long);
    static_assert(TB + 4 <= 64 * sizeof(uint32_t), "pinned word buffer too small");
    CKF(cudaMemcpyAsync(c->h_small, touched, TB, cudaMemcpyDeviceToHost, st));
    CKF(cudaMemcpyAsync(c->h_small + TB / 4, c->d_err, 4, cudaMemcpyDeviceToHost, st));
    CKF(cudaStreamSynchronize(st));
    unsigned long long tv[2 * (FEM_MAX_LEN + 1)];
    std::memcpy(tv, c->h_small, TB);
    const uint32_t e = c->h_small[TB / 4];
    for (fem_level_stats &ls : c->stats) {
        ls.touched_relaxed = tv[2 * ls.level];
        ls.touched_exact = tv[2 * ls.level + 1];
    }
    for (uint32_t N = 2; N <= max_len; ++N) {
        const uint32_t f = staged_f[N];
        if (!f) continue;
        const uint8_t *h = static_cast<const uint8_t *>(c->pin[N].p);
        res->eps[N - 1].resize(f);
        res->counts[N - 1].resize(f);
        std::memcpy(res->eps[N - 1].data(), h, (size_t)f * sizeof(fem_episode));
        std::memcpy(res->counts[N - 1].data(), h + (size_t)f * sizeof(fem_episode), (size_t)f * 4);
    }
    RETF(err_status(e));
    *out = res;
    return FEM_OK;
#undef RETF
#undef CKF
}

int fem_result_level(const fem_result *r, uint32_t level, uint32_t *m_out,
                     const fem_episode **eps, const uint32_t **counts) {
    if (!r || !m_out || level < 1 || level > r->eps.size()) return FEM_EINVAL;
    *m_out = (uint32_t)r->eps[level - 1].size();
    if (eps) *eps = r->eps[level - 1].data();
    if (counts) *counts = r->counts[level - 1].data();
    return FEM_OK;
}

uint32_t fem_result_max_level(const fem_result *r) {
    if (!r) return 0;
    uint32_t L = 0;
    for (uint32_t i = 0; i < r->eps.size(); ++i)
        if (!r->eps[i].empty()) L = i + 1;
    return L;
}

void fem_result_free(fem_result *r) { delete r; }

int fem_last_mine_stats(fem_ctx *c, fem_level_stats *out, uint32_t cap) {
    if (!c || (cap && !out)) return FEM_EINVAL;
    const uint32_t k = std::min<uint32_t>(cap, (uint32_t)c->stats.size());
    for (uint32_t i = 0; i < k; ++i) out[i] = c->stats[i];
    return (int)k;
}

}  // extern "C"

// ============================================================================ batches
namespace {

constexpr uint32_t kBatchChunksPerItem = 16;  // segment length of batched work items (rule)
constexpr uint32_t kBatchMinChunksPerItem = 8;  // shortest segment length tried when tuning
constexpr uint32_t kBatchMinThreads = 64;       // smallest block size tried when tuning

struct BatchGroup {
    int N = 0;
    uint32_t n_jobs = 0, m = 0;
    std::vector<uint32_t> user_job;  // user job index of each group job
    std::vector<uint32_t> off;       // host copy of cand_off
    fem_episode *cands = nullptr;
    uint32_t *cand_off = nullptr, *theta = nullptr;
    CountParams *rjobs = nullptr, *xjobs = nullptr;
    BatchOut *outs = nullptr;
    uint32_t *rel = nullptr, *ex = nullptr, *idx = nullptr, *scratch = nullptr;
    uint8_t *flags = nullptr, *redo = nullptr, *xredo = nullptr;
    uint32_t *item_off_r = nullptr, *item_off_x = nullptr;
    uint4 *items_r = nullptr, *items_x = nullptr;
    uint32_t cap_r = 0, cap_x = 0;
    uint32_t *counters = nullptr;  // n_items_r, n_items_x, queue_r, queue_x, n_idx
    uint4 *tables = nullptr;
    uint32_t SB = 0, Tr = 128, Tx = 128, Rx = 16;
    uint32_t cpi = kBatchChunksPerItem;  // chunks per work item (segment length)
    std::vector<uint32_t> nch, mj;       // per group job: stream chunks, candidates
    std::vector<CountParams> rj, xj;     // host templates of the per-job parameters
};

}  // namespace

struct fem_batch {
    fem_ctx *ctx = nullptr;
    std::vector<fem_job> jobs;
    std::vector<BatchGroup> groups;
    std::vector<void *> allocs;
    std::vector<size_t> alloc_bytes;
    uint2 *ivl = nullptr;
    uint32_t nI = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t graph_kernels = 0;  // kernel nodes of the captured graph (launch accounting)
};

namespace {

template <typename T>
int balloc(fem_batch *b, size_t count, T **out) {
    void *p = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 256);
    RET(cmalloc(b->ctx, &p, bytes));
    b->allocs.push_back(p);
    b->alloc_bytes.push_back(bytes);
    *out = static_cast<T *>(p);
    return FEM_OK;
}

void batch_free(fem_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (size_t i = 0; i < b->allocs.size(); ++i) cfree(b->ctx, b->allocs[i], b->alloc_bytes[i]);
    delete b;
}

// Set a group's launch shape: segment length (chunks per item) and block sizes of
// the two passes; rewrites the per-job segment counts and table slices.
int batch_shape(BatchGroup &g, uint32_t cpi, uint32_t Tr, uint32_t Tx, cudaStream_t st) {
    g.cpi = cpi, g.Tr = Tr, g.Tx = Tx;
    uint64_t toff = 0;
    for (uint32_t k = 0; k < g.n_jobs; ++k) {
        uint32_t P = (g.nch[k] + cpi - 1) / cpi;
        const uint32_t cps = (g.nch[k] + P - 1) / P;
        P = (g.nch[k] + cps - 1) / cps;
        for (CountParams *q : {&g.rj[k], &g.xj[k]}) {
            q->cps = cps;
            q->P = P;
            q->tables = g.tables + toff;
        }
        toff += (uint64_t)g.mj[k] * P * S_MAX;
    }
    CK(cudaMemcpyAsync(g.rjobs, g.rj.data(), g.n_jobs * sizeof(CountParams),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(g.xjobs, g.xj.data(), g.n_jobs * sizeof(CountParams),
                       cudaMemcpyHostToDevice, st));
    return FEM_OK;
}

// The two-pass count of one length group, enqueued on st without host round trips.
int batch_enqueue_group(fem_ctx *c, BatchGroup &g, cudaStream_t st) {
    {
        CK(cudaMemsetAsync(g.counters, 0, 8 * sizeof(uint32_t), st));
        CK(cudaMemsetAsync(g.redo, 0, g.m, st));
        CK(cudaMemsetAsync(g.xredo, 0, g.m, st));
        // first pass: relaxed counts of every candidate (Algorithm 3)
        CK(launch_batch_items(g.rjobs, g.n_jobs, g.Tr, g.item_off_r, g.counters + 0, g.cap_r,
                              g.items_r, st));
        CK(launch_count_batch(g.N, FEM_PASS_RELAXED, 1, g.Tr, g.rjobs, g.items_r, g.counters + 0,
                              g.counters + 2, g.SB, c->sm_count, st));
        CK(launch_stitch_batch(g.rjobs, g.cand_off, g.n_jobs, g.m, c->d_err, st));
        // elimination at each job's theta (Algorithm 4)
        CK(launch_batch_keep_flags(g.rel, g.cand_off, g.theta, g.n_jobs, g.m, g.flags, st));
        CK(launch_compact(nullptr, g.flags, 0, g.m, g.idx, g.counters + 4, g.scratch, st));
        // second pass: exact counts of the survivors (Algorithm 1)
        CK(launch_batch_exact_jobs(g.xjobs, g.cand_off, g.n_jobs, g.idx, g.counters + 4, g.ex, st));
        CK(launch_batch_items(g.xjobs, g.n_jobs, g.Tx, g.item_off_x, g.counters + 1, g.cap_x,
                              g.items_x, st));
        CK(launch_count_batch(g.N, FEM_PASS_EXACT, g.Rx, g.Tx, g.xjobs, g.items_x, g.counters + 1,
                              g.counters + 3, g.SB, c->sm_count, st));
        CK(launch_stitch_batch(g.xjobs, g.cand_off, g.n_jobs, g.m, c->d_err, st));
        CK(launch_batch_outputs(g.outs, g.cand_off, g.n_jobs, g.m, g.idx, g.counters + 4, g.ex, st));
    }
    return FEM_OK;
}

// The whole two-pass count of the batch, enqueued on st without host round trips.
int batch_enqueue(fem_batch *b, cudaStream_t st) {
    for (BatchGroup &g : b->groups) RET(batch_enqueue_group(b->ctx, g, st));
    return FEM_OK;
}

// Batch launch shapes by measurement: for each length group, time every segment
// length (8, 16, 32 chunks per item) and block size pair, each a complete two-pass
// count, and keep the fastest.
int batch_tune(fem_batch *b, cudaStream_t st) {
    fem_ctx *c = b->ctx;
    for (BatchGroup &g : b->groups) {
        float best = -1;
        uint32_t bc = g.cpi, br = g.Tr, bx = g.Tx;
        for (uint32_t cpi : {8u, 16u, 32u}) {
            for (uint32_t Tr : {128u, 256u}) {
                if (Tr == 256 && g.N > 3) continue;
                for (uint32_t Tx : {64u, 128u}) {
                    RET(batch_shape(g, cpi, Tr, Tx, st));
                    float ms = -1;
                    for (int rep = 0; rep < 2; ++rep) {  // the faster of two (kernel loading)
                        CK(cudaMemsetAsync(c->d_err, 0, 4, st));
                        CK(cudaEventRecord(c->tev[0], st));
                        RET(batch_enqueue_group(c, g, st));
                        CK(cudaEventRecord(c->tev[1], st));
                        uint32_t e;
                        RET(read_err(c, st, &e));
                        RET(err_status(e));
                        float t = 0;
                        CK(cudaEventElapsedTime(&t, c->tev[0], c->tev[1]));
                        if (e & ERR_CAP) t *= 4;  // needs recounts
                        if (ms < 0 || t < ms) ms = t;
                    }
                    if (best < 0 || ms < best) best = ms, bc = cpi, br = Tr, bx = Tx;
                }
            }
        }
        RET(batch_shape(g, bc, br, bx, st));
        if (std::getenv("FEM_DEBUG"))
            std::fprintf(stderr, "fem: batch N=%d jobs=%u m=%u: %u chunks per item, T %u/%u, %.3f ms\n",
                         g.N, g.n_jobs, g.m, bc, br, bx, best);
    }
    return FEM_OK;
}

}  // namespace

extern "C" {

int fem_batch_create(fem_ctx *c, const fem_job *jobs, uint32_t n_jobs, const fem_interval *I,
                     uint32_t nI, void *cuda_stream, fem_batch **out) {
    if (!c || !out || !jobs || n_jobs == 0) return FEM_EINVAL;
    *out = nullptr;
    for (uint32_t j = 0; j < n_jobs; ++j) {
        const StreamDev *s = find_stream(c, jobs[j].stream_id);
        if (!s) return FEM_ENOSTREAM;
        if (jobs[j].len < 1 || jobs[j].len > FEM_MAX_LEN) return FEM_EINVAL;
        if (jobs[j].m && (!jobs[j].cands || !jobs[j].exact_out || !jobs[j].survived_out))
            return FEM_EINVAL;
        RET(check_intervals(*s, I, nI));
    }
    cudaSetDevice(c->device);
    cudaStream_t st = pick(c, cuda_stream);
    fem_batch *b = new (std::nothrow) fem_batch;
    if (!b) return FEM_ENOMEM;
    b->ctx = c;
    b->jobs.assign(jobs, jobs + n_jobs);
    b->nI = nI;
    auto fail = [&](int rc) {
        cudaStreamSynchronize(st);
        batch_free(b);
        return rc;
    };
#define BRET(x)                           \
    do {                                  \
        int r_ = (x);                     \
        if (r_ != FEM_OK) return fail(r_); \
    } while (0)
#define BCK(x)                                          \
    do {                                                \
        if ((x) != cudaSuccess) return fail(FEM_ECUDA); \
    } while (0)
    BRET(balloc(b, std::max<uint32_t>(nI, 1), &b->ivl));
    if (nI) BCK(cudaMemcpyAsync(b->ivl, I, nI * sizeof(uint2), cudaMemcpyHostToDevice, st));

    for (int N = 1; N <= FEM_MAX_LEN; ++N) {
        BatchGroup g;
        g.N = N;
        struct Ent {
            uint32_t j, nch;
        };
        std::vector<Ent> ents;
        for (uint32_t j = 0; j < n_jobs; ++j) {
            if ((int)jobs[j].len != N || jobs[j].m == 0) continue;
            const StreamDev &s = *find_stream(c, jobs[j].stream_id);
            ents.push_back({j, std::max<uint32_t>(s.n_chunks, 1)});
        }
        if (ents.empty()) continue;
        // longest streams first: with equal segment lengths their items are the
        // longest, and the persistent blocks then finish together
        std::stable_sort(ents.begin(), ents.end(),
                         [](const Ent &a, const Ent &b2) { return a.nch > b2.nch; });
        g.n_jobs = (uint32_t)ents.size();
        g.Tr = N <= 3 ? 256 : 128;
        g.Tx = 128;
        g.Rx = 16;
        // capacities for every shape batch_shape may set (shortest segments, smallest
        // blocks)
        uint64_t m = 0, tab = 0, cap = 0;
        uint32_t max_offs = 8;
        g.off.push_back(0);
        for (const Ent &e : ents) {
            const fem_job &jb = jobs[e.j];
            g.user_job.push_back(e.j);
            g.nch.push_back(e.nch);
            g.mj.push_back(jb.m);
            m += jb.m;
            g.off.push_back((uint32_t)m);
            const uint64_t Pmax = (e.nch + kBatchMinChunksPerItem - 1) / kBatchMinChunksPerItem;
            tab += (uint64_t)jb.m * Pmax * S_MAX;
            cap += (uint64_t)((jb.m + kBatchMinThreads - 1) / kBatchMinThreads) * Pmax;
            max_offs = std::max(max_offs, find_stream(c, jb.stream_id)->offs);
        }
        const uint64_t cap_r = cap, cap_x = cap;
        if (m > 0xFFFFFFF0ull || cap_r > 0xFFFFFFF0ull) return fail(FEM_ENOMEM);
        g.m = (uint32_t)m;
        g.cap_r = (uint32_t)cap_r;
        g.cap_x = (uint32_t)cap_x;
        g.SB = stage_bytes(max_offs);
        const uint32_t n = g.n_jobs;
        BRET(balloc(b, m, &g.cands));
        BRET(balloc(b, n + 1, &g.cand_off));
        BRET(balloc(b, n, &g.theta));
        BRET(balloc(b, n, &g.rjobs));
        BRET(balloc(b, n, &g.xjobs));
        BRET(balloc(b, n, &g.outs));
        BRET(balloc(b, m, &g.rel));
        BRET(balloc(b, m, &g.ex));
        BRET(balloc(b, m, &g.idx));
        BRET(balloc(b, compact_scratch_words(g.m), &g.scratch));
        BRET(balloc(b, m, &g.flags));
        BRET(balloc(b, m, &g.redo));
        BRET(balloc(b, m, &g.xredo));
        BRET(balloc(b, n + 1, &g.item_off_r));
        BRET(balloc(b, n + 1, &g.item_off_x));
        BRET(balloc(b, cap_r, &g.items_r));
        BRET(balloc(b, cap_x, &g.items_x));
        BRET(balloc(b, 8, &g.counters));
        BRET(balloc(b, tab, &g.tables));
        std::vector<CountParams> &rj = g.rj, &xj = g.xj;
        rj.resize(n);
        xj.resize(n);
        std::vector<uint32_t> th(n);
        std::vector<BatchOut> bo(n);
        for (uint32_t k = 0; k < n; ++k) {
            const fem_job &jb = jobs[ents[k].j];
            const StreamDev &s = *find_stream(c, jb.stream_id);
            BCK(cudaMemcpyAsync(g.cands + g.off[k], jb.cands, (size_t)jb.m * sizeof(fem_episode),
                                cudaMemcpyDeviceToDevice, st));
            CountParams p{};
            p.bev = s.bev;
            p.boff = s.boff;
            p.cfirst = s.cfirst;
            p.t = s.t;
            p.offs = s.offs;
            p.n_chunks = s.n_chunks;
            p.n = s.n;
            p.K = s.K;
            p.ivl = b->ivl;
            p.n_ivl = nI;
            p.err = c->d_err;  // segments and tables: batch_shape
            CountParams r = p, x = p;
            r.cands = g.cands + g.off[k];
            r.m = jb.m;
            r.out = g.rel + g.off[k];
            r.redo = g.redo + g.off[k];
            x.cands = g.cands;  // gathered through the survivor list at run time
            x.m = 0;
            x.redo = g.xredo + g.off[k];
            rj[k] = r;
            xj[k] = x;
            th[k] = jb.theta;
            bo[k] = BatchOut{jb.exact_out, jb.survived_out};
        }
        BRET(batch_shape(g, kBatchChunksPerItem, g.Tr, g.Tx, st));
        BCK(cudaMemcpyAsync(g.cand_off, g.off.data(), (n + 1) * 4, cudaMemcpyHostToDevice, st));
        BCK(cudaMemcpyAsync(g.theta, th.data(), n * 4, cudaMemcpyHostToDevice, st));
        BCK(cudaMemcpyAsync(g.outs, bo.data(), n * sizeof(BatchOut), cudaMemcpyHostToDevice, st));
        BCK(cudaStreamSynchronize(st));  // host staging vectors go out of scope
        b->groups.push_back(std::move(g));
    }
    // measured shapes when tuning is on; one eager run (sets kernel attributes, checks
    // the inputs); then capture
    if (c->tune_on) BRET(batch_tune(b, st));
    BRET(fem_batch_run(b, cuda_stream));
    BCK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = batch_enqueue(b, b->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &graph);
    if (rc != FEM_OK) return fail(rc);
    if (ce != cudaSuccess) return fail(FEM_ECUDA);
    b->graph = graph;
    BCK(cudaGraphInstantiate(&b->exec, graph, 0));
    size_t n_nodes = 0;
    BCK(cudaGraphGetNodes(graph, nullptr, &n_nodes));
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    if (n_nodes) BCK(cudaGraphGetNodes(graph, nodes.data(), &n_nodes));
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        BCK(cudaGraphNodeGetType(nd, &ty));
        b->graph_kernels += ty == cudaGraphNodeTypeKernel;
    }
    *out = b;
    return FEM_OK;
#undef BRET
#undef BCK
}

int fem_batch_run(fem_batch *b, void *cuda_stream) {
    if (!b) return FEM_EINVAL;
    fem_ctx *c = b->ctx;
    cudaSetDevice(c->device);
    cudaStream_t st = pick(c, cuda_stream);
    CK(cudaMemsetAsync(c->d_err, 0, 4, st));
    if (b->exec) {
        CK(cudaGraphLaunch(b->exec, st));
        note_launch(b->graph_kernels);
    } else {
        RET(batch_enqueue(b, st));
    }
    uint32_t e;
    RET(read_err(c, st, &e));
    RET(err_status(e));
    if (!(e & ERR_CAP)) return FEM_OK;
    // A capacity guard tripped somewhere: recount the affected jobs one at a time
    // with the single-recording path, which widens rings as needed.
    std::vector<fem_interval> I(b->nI);
    if (b->nI) CK(cudaMemcpy(I.data(), b->ivl, b->nI * sizeof(uint2), cudaMemcpyDeviceToHost));
    for (BatchGroup &g : b->groups) {
        std::vector<uint8_t> r(g.m), x(g.m);
        CK(cudaMemcpy(r.data(), g.redo, g.m, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(x.data(), g.xredo, g.m, cudaMemcpyDeviceToHost));
        for (uint32_t k = 0; k < g.n_jobs; ++k) {
            bool hit = false;
            for (uint32_t i = g.off[k]; i < g.off[k + 1] && !hit; ++i) hit = r[i] || x[i];
            if (!hit) continue;
            const fem_job &jb = b->jobs[g.user_job[k]];
            RET(fem_count_two_pass(c, jb.stream_id, jb.cands, jb.m, 1, I.data(), b->nI, jb.theta,
                                   jb.exact_out, jb.survived_out, 1, st));
        }
    }
    return FEM_OK;
}

int fem_batch_destroy(fem_batch *b) {
    if (!b) return FEM_EINVAL;
    cudaSetDevice(b->ctx->device);
    cudaDeviceSynchronize();
    batch_free(b);
    return FEM_OK;
}

}  // extern "C"
