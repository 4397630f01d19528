// fem_serve.cu -- near-real-time serving over growing streams (include/fem.h,
// "Serving").  Continuous batching: a request is admitted while others run when
// its device memory fits the server's arena and a slot is free; its whole work is
// enqueued at once on one of several CUDA streams, so admitted requests overlap on
// the device, and its memory returns to the arena as soon as its results have
// been copied to pinned host memory.
//
// Ordering: appending events regroups the stream's last (partial) chunk in place.
// Every request waits (cudaStreamWaitEvent) for the append that preceded its
// submission, and an append waits for the requests still reading that partial
// chunk, so a reader never sees a chunk being rewritten.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "fem_internal.cuh"

using namespace fem;

namespace {

// First-fit allocator over one pre-reserved block (device or pinned host memory).
struct Arena {
    char *base = nullptr;
    size_t size = 0, used = 0;
    bool pinned = false;
    std::map<size_t, size_t> free_;  // offset -> length

    bool init(size_t bytes, bool host_pinned) {
        pinned = host_pinned;
        void *p = nullptr;
        const cudaError_t e = host_pinned ? cudaMallocHost(&p, bytes) : cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        base = static_cast<char *>(p);
        size = bytes;
        free_[0] = bytes;
        return true;
    }
    void destroy() {
        if (base) (pinned ? cudaFreeHost(base) : cudaFree(base));
        base = nullptr;
    }
    static size_t round(size_t b) { return (b + 255) & ~(size_t)255; }
    void *alloc(size_t bytes) {
        bytes = round(std::max<size_t>(bytes, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > bytes) free_[off + bytes] = len - bytes;
            used += bytes;
            return base + off;
        }
        return nullptr;
    }
    void release(void *p, size_t bytes) {
        if (!p) return;
        bytes = round(std::max<size_t>(bytes, 1));
        size_t off = static_cast<char *>(p) - base;
        used -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
};

struct ServeStream {
    StreamDev s;
    uint64_t cap_events = 0;
    std::vector<uint32_t> t_host;  // times appended so far (window starts are found here)
    cudaEvent_t ingested = nullptr;
    std::vector<cudaEvent_t> tail_readers;  // work reading the current partial chunk
};

// One length group of a request's candidates (contiguous after sorting by length).
struct Group {
    uint32_t N = 0, off = 0, m = 0;
    uint32_t stride = 0;  // carried-state words per candidate (standing)
};

struct Request {
    uint64_t id = 0;
    int32_t sid = 0;
    int mode = 0;
    uint32_t m = 0, theta = 0, nI = 0;
    uint64_t ev_begin = 0, ev_end = 0;  // events covered by the latest result
    std::vector<Group> groups;
    std::vector<uint32_t> perm;  // caller's candidate c sits at sorted position perm[c]
    // device block
    char *dblk = nullptr;
    size_t dbytes = 0;
    fem_episode *cands = nullptr;
    uint2 *ivl = nullptr;
    uint32_t *rel = nullptr, *idx = nullptr, *ex = nullptr, *out = nullptr, *scratch = nullptr;
    uint32_t *cnt = nullptr, *err = nullptr, *state = nullptr;
    uint8_t *flags = nullptr, *redo = nullptr;
    uint4 *tables = nullptr;     // MapConcatenate transfer tables of a one-shot relaxed pass
    uint64_t tab_items = 0;      // (episode, segment) pairs the tables hold
    // pinned host block: out (m), flags (m), err (1), staging of candidates
    char *hblk = nullptr;
    size_t hbytes = 0;
    uint32_t *h_out = nullptr, *h_err = nullptr;
    uint8_t *h_flags = nullptr;
    fem_episode *h_cands = nullptr;
    cudaStream_t lane = nullptr;
    cudaEvent_t done = nullptr;
    bool in_flight = false, fresh = false, holds_slot = false;
    int status = FEM_OK;
    uint64_t first_event = 0;            // a standing request counts from here
    std::vector<uint32_t> pub_counts;    // latest finished result, sorted order
    std::vector<uint8_t> pub_flags;
    uint64_t pub_begin = 0, pub_end = 0;
};

constexpr uint32_t kServeRing = 16;  // exact-pass clusters per node in serving
// A one-shot request's passes give each length group about this many threads per SM
// through MapConcatenate segments (a 1k-candidate group alone would fill a few SMs), as
// the context's counts do; the transfer tables are part of the request's device memory.
constexpr uint32_t kServeThreadsPerSM = 2048;

// Segments of a one-shot pass over nch chunks for m candidates (1: none).  The tables
// of one request may take an eighth of the arena at most.
uint32_t oneshot_segments(uint32_t m, uint32_t nch, int sm_count, size_t arena_bytes) {
    if (m == 0 || nch < 2) return 1;
    const uint64_t target = (uint64_t)sm_count * kServeThreadsPerSM;
    uint64_t P = std::min<uint64_t>((target + m - 1) / m, nch);
    const uint64_t cap = arena_bytes / 8 / (S_MAX * sizeof(uint4)) / m;
    P = std::min<uint64_t>(P, cap);
    return P < 2 ? 1u : (uint32_t)P;
}

}  // namespace

struct fem_server {
    fem_ctx *ctx = nullptr;
    int device = 0;
    fem_server_config cfg{};
    Arena dev, host;
    std::vector<cudaStream_t> lanes;
    uint32_t next_lane = 0;
    cudaStream_t ingest = nullptr;
    std::map<int32_t, ServeStream> streams;
    int32_t next_sid = 1;
    std::map<uint64_t, Request> reqs;
    uint64_t next_req = 1;
    uint32_t active = 0;
    std::vector<cudaEvent_t> event_pool;
    struct Staged {
        void *p;
        size_t bytes;
        cudaEvent_t e;
    };
    std::vector<Staged> staged;  // pinned copies of appended chunks still being uploaded
};

namespace {

#define SCK(x)                                   \
    do {                                         \
        if ((x) != cudaSuccess) {                \
            cudaGetLastError();                  \
            return FEM_ECUDA;                    \
        }                                        \
    } while (0)
#define SRET(x)                      \
    do {                             \
        int r_ = (x);                \
        if (r_ != FEM_OK) return r_; \
    } while (0)

cudaEvent_t take_event(fem_server *v) {
    if (!v->event_pool.empty()) {
        cudaEvent_t e = v->event_pool.back();
        v->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

CountParams base_params(const StreamDev &s, const Request &r, const Group &g, int pass) {
    CountParams p{};
    p.bev = s.bev;
    p.boff = s.boff;
    p.cfirst = s.cfirst;
    p.t = s.t;
    p.offs = s.offs;
    p.n_chunks = s.n_chunks;
    p.n = s.n;
    p.K = s.K;
    p.ivl = r.ivl;
    p.n_ivl = r.nI;
    p.cps = std::max<uint32_t>(s.n_chunks, 1);
    p.P = 1;
    p.redo = r.redo + g.off;
    p.err = r.err;
    p.ranged = 1;
    p.ev_begin = r.ev_begin;
    p.ev_end = r.ev_end;
    (void)pass;
    return p;
}

uint32_t serve_threads(int N, int pass, uint32_t R, uint32_t offs, bool mc = false,
                       uint32_t classes = S_MAX) {
    for (uint32_t T : {128u, 64u, 32u})
        if (count_smem_bytes(N, pass, mc, R, T, offs, classes) <= 100 * 1024) return T;
    return 32;
}

// One-shot: Algorithm 4 over [ev_begin, ev_end) of the stream, per length group,
// with every size on the device (no host round trip).  A group of few candidates runs
// both passes over MapConcatenate segments of the range (the exact pass over the
// survivors, whose number stays on the device).  attempt 0: the rule's segments, 8
// entry classes per table, exact lists of kServeRing clusters; attempt 1 (after a
// capacity guard tripped): a quarter of the segments with 32 classes per table in the
// same memory and lists of 32 clusters; attempt 2: one segment, lists of 128.
int enqueue_oneshot(fem_server *v, Request &r, const StreamDev &s, int attempt) {
    cudaStream_t st = r.lane;
    const uint32_t cr0 = (uint32_t)(r.ev_begin / CHUNK);
    const uint32_t cr1 = (uint32_t)((r.ev_end + CHUNK - 1) / CHUNK);
    const uint32_t nch = cr1 > cr0 ? cr1 - cr0 : 0u;
    const uint32_t R = attempt == 0 ? kServeRing : attempt == 1 ? 32u : 128u;
    const uint32_t cls = attempt == 0 ? S_MAX : S_RECOUNT;
    // the stitch skips episodes flagged for a recount: no flag may survive from the
    // memory's last user
    SCK(cudaMemsetAsync(r.redo, 0, r.m, st));
    for (const Group &g : r.groups) {
        CountParams p = base_params(s, r, g, FEM_PASS_RELAXED);
        p.cands = r.cands + g.off;
        p.m = g.m;
        p.out = r.rel + g.off;
        uint32_t P = attempt < 2 && r.tables
                         ? oneshot_segments(g.m, nch, fem_ctx_sms(v->ctx), v->cfg.mem_budget_bytes)
                         : 1u;
        if (attempt == 1) P /= S_RECOUNT / S_MAX;  // the same table memory, 4x the slots
        if (P > 1) {
            const uint32_t cps = (nch + P - 1) / P;
            P = (nch + cps - 1) / cps;
            if ((uint64_t)P * g.m * cls > r.tab_items * S_MAX) P = 1;
            if (P > 1) {
                p.cps = cps;
                p.P = P;
                p.tables = r.tables;
            }
        }
        const uint32_t pcls = P > 1 ? cls : S_MAX;
        SCK(launch_count(g.N, FEM_PASS_RELAXED, P > 1, 1,
                         serve_threads(g.N, FEM_PASS_RELAXED, 1, s.offs, P > 1, pcls), p, st,
                         pcls));
        if (P > 1)
            SCK(launch_stitch(r.tables, g.m, P, r.rel + g.off, r.redo + g.off, r.err, st, pcls));
        SCK(launch_compact(r.rel + g.off, nullptr, r.theta, g.m, r.idx + g.off,
                           r.cnt + (&g - r.groups.data()), r.scratch, st));
        // the exact pass over the survivors (their number stays on the device): a grid for
        // all g.m, the blocks past the survivors leave at once; with the relaxed pass's
        // segments, so that a few survivors still spread over the GPU.  The stitch runs
        // over g.m slots too; those past the survivors hold the relaxed pass's tables and
        // their results are never scattered.
        CountParams x = base_params(s, r, g, FEM_PASS_EXACT);
        x.cands = r.cands + g.off;
        x.gather = r.idx + g.off;
        x.m = g.m;
        x.m_dev = r.cnt + (&g - r.groups.data());
        x.out = r.ex + g.off;
        const bool xmc = P > 1 && count_config_supported(g.N, FEM_PASS_EXACT, true, R);
        if (xmc) {
            x.cps = p.cps;
            x.P = P;
            x.tables = r.tables;
        }
        SCK(launch_count(g.N, FEM_PASS_EXACT, xmc, R,
                         serve_threads(g.N, FEM_PASS_EXACT, R, s.offs, xmc, pcls), x, st,
                         xmc ? pcls : S_MAX));
        if (xmc)
            SCK(launch_stitch(r.tables, g.m, P, r.ex + g.off, r.redo + g.off, r.err, st, pcls));
        SCK(cudaMemsetAsync(r.out + g.off, 0, (size_t)g.m * 4, st));
        SCK(cudaMemsetAsync(r.flags + g.off, 0, g.m, st));
        SCK(launch_scatter_dev(r.ex + g.off, r.idx + g.off, x.m_dev, g.m, r.out + g.off,
                               r.flags + g.off, st));
    }
    return FEM_OK;
}

// Standing: exact counts of every candidate, resumed from the carried state over
// the new events [ev_begin, ev_end).
int enqueue_standing(fem_server *v, Request &r, const StreamDev &s) {
    cudaStream_t st = r.lane;
    uint64_t soff = 0;
    for (const Group &g : r.groups) {
        CountParams x = base_params(s, r, g, FEM_PASS_EXACT);
        x.cands = r.cands + g.off;
        x.m = g.m;
        x.out = r.out + g.off;
        x.state = r.state + soff;
        x.state_stride = g.stride;
        SCK(launch_count(g.N, FEM_PASS_EXACT, false, kServeRing,
                         serve_threads(g.N, FEM_PASS_EXACT, kServeRing, s.offs), x, st));
        soff += (uint64_t)g.m * g.stride;
    }
    (void)v;
    return FEM_OK;
}

// Copy results to pinned memory, mark completion, register as a reader of the
// stream's partial chunk when the range ends inside it.
int finish_enqueue(fem_server *v, Request &r, ServeStream &ss) {
    cudaStream_t st = r.lane;
    SCK(cudaMemcpyAsync(r.h_out, r.out, (size_t)r.m * 4, cudaMemcpyDeviceToHost, st));
    if (r.mode == FEM_REQ_ONESHOT)
        SCK(cudaMemcpyAsync(r.h_flags, r.flags, r.m, cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(r.h_err, r.err, 4, cudaMemcpyDeviceToHost, st));
    if (!r.done) r.done = take_event(v);
    if (!r.done) return FEM_ECUDA;
    SCK(cudaEventRecord(r.done, st));
    if (r.ev_end % CHUNK) {
        cudaEvent_t e = take_event(v);
        if (!e) return FEM_ECUDA;
        SCK(cudaEventRecord(e, st));
        ss.tail_readers.push_back(e);
    }
    r.in_flight = true;
    return FEM_OK;
}

// Return pinned staging buffers whose uploads have finished (all of them if wait).
void reap_staging(fem_server *v, bool wait) {
    std::vector<fem_server::Staged> keep;
    for (auto &st : v->staged) {
        if (wait) cudaEventSynchronize(st.e);
        if (cudaEventQuery(st.e) == cudaSuccess) {
            v->host.release(st.p, st.bytes);
            v->event_pool.push_back(st.e);
        } else {
            cudaGetLastError();
            keep.push_back(st);
        }
    }
    v->staged.swap(keep);
}

void release_memory(fem_server *v, Request &r) {
    if (r.dblk) v->dev.release(r.dblk, r.dbytes);
    r.dblk = nullptr;
}

}  // namespace

extern "C" {

int fem_server_create(fem_ctx *ctx, const fem_server_config *cfg, fem_server **out) {
    if (!ctx || !out) return FEM_EINVAL;
    *out = nullptr;
    fem_server *v = new (std::nothrow) fem_server;
    if (!v) return FEM_ENOMEM;
    v->ctx = ctx;
    v->device = fem_ctx_device(ctx);
    if (cfg) v->cfg = *cfg;
    if (!v->cfg.mem_budget_bytes) v->cfg.mem_budget_bytes = (size_t)1 << 30;
    if (!v->cfg.max_active) v->cfg.max_active = 64;
    if (!v->cfg.n_lanes) v->cfg.n_lanes = 8;
    cudaSetDevice(v->device);
    bool ok = v->dev.init(v->cfg.mem_budget_bytes, false) &&
              v->host.init(std::max<size_t>(v->cfg.mem_budget_bytes / 4, (size_t)64 << 20), true) &&
              cudaStreamCreateWithFlags(&v->ingest, cudaStreamNonBlocking) == cudaSuccess;
    for (uint32_t i = 0; ok && i < v->cfg.n_lanes; ++i) {
        cudaStream_t s = nullptr;
        ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) v->lanes.push_back(s);
    }
    if (!ok) {
        cudaGetLastError();
        fem_server_destroy(v);
        return FEM_ENOMEM;
    }
    *out = v;
    return FEM_OK;
}

int fem_server_destroy(fem_server *v) {
    if (!v) return FEM_EINVAL;
    cudaSetDevice(v->device);
    cudaDeviceSynchronize();
    for (auto &kv : v->reqs)
        if (kv.second.done) cudaEventDestroy(kv.second.done);
    for (auto &kv : v->streams) {
        StreamDev &s = kv.second.s;
        cudaFree(s.t);
        cudaFree(s.type);
        cudaFree(s.bev);
        cudaFree(s.boff);
        cudaFree(s.cfirst);
        if (kv.second.ingested) cudaEventDestroy(kv.second.ingested);
        for (cudaEvent_t e : kv.second.tail_readers) cudaEventDestroy(e);
    }
    for (cudaEvent_t e : v->event_pool) cudaEventDestroy(e);
    for (cudaStream_t s : v->lanes) cudaStreamDestroy(s);
    if (v->ingest) cudaStreamDestroy(v->ingest);
    v->dev.destroy();
    v->host.destroy();
    delete v;
    return FEM_OK;
}

int fem_server_open_stream(fem_server *v, uint32_t K, uint64_t cap, int32_t *sid_out) {
    if (!v || !sid_out || K == 0 || K > FEM_MAX_TYPES || cap == 0 || cap >= 0xFFFFFFF0ull)
        return FEM_EINVAL;
    cudaSetDevice(v->device);
    ServeStream ss;
    StreamDev &s = ss.s;
    s.K = K;
    s.offs = offs_stride(K);
    const uint64_t nc = (cap + CHUNK - 1) / CHUNK;
    ss.cap_events = nc * CHUNK;
    bool ok = cudaMalloc(&s.t, ss.cap_events * 4) == cudaSuccess &&
              cudaMalloc(&s.type, ss.cap_events) == cudaSuccess &&
              cudaMalloc(&s.bev, ss.cap_events * 8) == cudaSuccess &&
              cudaMalloc(&s.boff, nc * s.offs * 2) == cudaSuccess &&
              cudaMalloc(&s.cfirst, (nc + 1) * 4) == cudaSuccess &&
              cudaEventCreateWithFlags(&ss.ingested, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaFree(s.t);
        cudaFree(s.type);
        cudaFree(s.bev);
        cudaFree(s.boff);
        cudaFree(s.cfirst);
        return FEM_ENOMEM;
    }
    SCK(cudaEventRecord(ss.ingested, v->ingest));
    const int32_t id = v->next_sid++;
    v->streams[id] = std::move(ss);
    *sid_out = id;
    return FEM_OK;
}

int fem_server_append(fem_server *v, int32_t sid, const uint8_t *types, const uint32_t *t_us,
                      uint32_t n) {
    if (!v || (n && (!types || !t_us))) return FEM_EINVAL;
    auto it = v->streams.find(sid);
    if (it == v->streams.end()) return FEM_ENOSTREAM;
    ServeStream &ss = it->second;
    StreamDev &s = ss.s;
    if (n == 0) return FEM_OK;
    if (s.n + n > ss.cap_events) return FEM_ENOMEM;
    uint32_t prev = ss.t_host.empty() ? 0u : ss.t_host.back();
    for (uint32_t i = 0; i < n; ++i) {
        if (types[i] >= s.K) return FEM_ETYPE;
        if (t_us[i] < prev) return FEM_EUNSORTED;
        prev = t_us[i];
    }
    cudaSetDevice(v->device);
    // the partial chunk is rewritten: wait for the work still reading it
    for (cudaEvent_t e : ss.tail_readers) {
        SCK(cudaStreamWaitEvent(v->ingest, e, 0));
        v->event_pool.push_back(e);
    }
    ss.tail_readers.clear();
    // stage the chunk in pinned memory so the upload never blocks the caller
    const size_t sb = (size_t)n * 5;
    char *hs = static_cast<char *>(v->host.alloc(sb));
    if (!hs) {
        reap_staging(v, false);
        hs = static_cast<char *>(v->host.alloc(sb));
    }
    if (!hs) {
        reap_staging(v, true);
        hs = static_cast<char *>(v->host.alloc(sb));
    }
    if (!hs) return FEM_ENOMEM;
    std::memcpy(hs, t_us, (size_t)n * 4);
    std::memcpy(hs + (size_t)n * 4, types, n);
    const uint64_t n_old = s.n;
    SCK(cudaMemcpyAsync(s.t + n_old, hs, (size_t)n * 4, cudaMemcpyHostToDevice, v->ingest));
    SCK(cudaMemcpyAsync(s.type + n_old, hs + (size_t)n * 4, n, cudaMemcpyHostToDevice, v->ingest));
    cudaEvent_t se = take_event(v);
    if (!se) return FEM_ECUDA;
    SCK(cudaEventRecord(se, v->ingest));
    v->staged.push_back({hs, sb, se});
    s.n = n_old + n;
    s.n_chunks = (uint32_t)((s.n + CHUNK - 1) / CHUNK);
    s.t_max = prev;
    SCK(launch_bucket_chunks(s, (uint32_t)(n_old / CHUNK), s.n_chunks, v->ingest));
    SCK(cudaEventRecord(ss.ingested, v->ingest));
    ss.t_host.insert(ss.t_host.end(), t_us, t_us + n);
    return FEM_OK;
}

namespace {
constexpr uint32_t kServeMaxHi = 1u << 26;     // interval bound accepted by the server (67 s)
constexpr uint32_t kServeMaxTime = 0xFFFFFFFFu - (1u << 26) - 2u;
}  // namespace

int fem_server_submit(fem_server *v, int32_t sid, const fem_episode *cands, uint32_t m,
                      const fem_interval *I, uint32_t nI, uint32_t theta, int mode,
                      uint32_t window_us, uint64_t *req_out) {
    if (!v || !req_out || m == 0 || !cands || (nI && !I) || nI > FEM_MAX_INTERVALS)
        return FEM_EINVAL;
    if (mode != FEM_REQ_ONESHOT && mode != FEM_REQ_STANDING) return FEM_EINVAL;
    auto it = v->streams.find(sid);
    if (it == v->streams.end()) return FEM_ENOSTREAM;
    ServeStream &ss = it->second;
    StreamDev &s = ss.s;
    for (uint32_t i = 0; i < nI; ++i)
        if (I[i].lo_us >= I[i].hi_us || I[i].hi_us > kServeMaxHi) return FEM_EINVAL;
    // candidates grouped by length, stable (a counting sort over the eight lengths)
    uint32_t by_len[FEM_MAX_LEN + 2] = {};
    for (uint32_t c = 0; c < m; ++c) {
        const fem_episode &e = cands[c];
        if (e.len < 1 || e.len > FEM_MAX_LEN) return FEM_EINVAL;
        for (uint32_t k = 0; k < e.len; ++k)
            if (e.types[k] >= s.K) return FEM_EINVAL;
        for (uint32_t k = 0; k + 1 < e.len; ++k)
            if (e.ivl[k] >= nI) return FEM_EINVAL;
        ++by_len[e.len + 1];
    }
    if (v->active >= v->cfg.max_active) return FEM_EADMIT;
    for (uint32_t N = 1; N <= FEM_MAX_LEN + 1; ++N) by_len[N] += by_len[N - 1];
    std::vector<uint32_t> order(m);
    for (uint32_t c = 0; c < m; ++c) order[by_len[cands[c].len]++] = c;
    Request r;
    r.id = v->next_req;
    r.sid = sid;
    r.mode = mode;
    r.m = m;
    r.theta = theta;
    r.nI = nI;
    r.perm.assign(m, 0);
    for (uint32_t pos = 0; pos < m; ++pos) {
        r.perm[order[pos]] = pos;
        const uint32_t N = cands[order[pos]].len;
        if (r.groups.empty() || r.groups.back().N != N) {
            Group g;
            g.N = N;
            g.off = pos;
            g.stride = 1 + (N - 1) * (1 + 2 * kServeRing);
            r.groups.push_back(g);
        }
        r.groups.back().m++;
    }
    // one device block: candidates, intervals, per-pass arrays, scratch, state
    uint32_t gmax = 0;
    uint64_t state_words = 0;
    for (const Group &g : r.groups) {
        gmax = std::max(gmax, g.m);
        state_words += (uint64_t)g.m * g.stride;
    }
    auto rnd = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // a one-shot request covers the last window_us of the stream as it is now
    r.ev_end = s.n;
    if (mode == FEM_REQ_ONESHOT) {
        r.ev_begin = 0;
        if (window_us && !ss.t_host.empty() && ss.t_host.back() >= window_us) {
            const uint32_t t0 = ss.t_host.back() - window_us;
            r.ev_begin = std::lower_bound(ss.t_host.begin(), ss.t_host.end(), t0) - ss.t_host.begin();
        }
        const uint32_t nch = (uint32_t)((r.ev_end + CHUNK - 1) / CHUNK - r.ev_begin / CHUNK);
        for (const Group &g : r.groups) {
            const uint32_t P =
                oneshot_segments(g.m, nch, fem_ctx_sms(v->ctx), v->cfg.mem_budget_bytes);
            if (P > 1) r.tab_items = std::max<uint64_t>(r.tab_items, (uint64_t)P * g.m);
        }
    }
    const size_t b_cands = rnd((size_t)m * 16), b_ivl = rnd(std::max<uint32_t>(nI, 1) * 8),
                 b_u32 = rnd((size_t)m * 4), b_u8 = rnd(m),
                 b_scr = rnd(compact_scratch_words(gmax) * 4), b_cnt = rnd(r.groups.size() * 4 + 4),
                 b_state = mode == FEM_REQ_STANDING ? rnd(state_words * 4) : 0,
                 b_tab = rnd(r.tab_items * S_MAX * sizeof(uint4));
    r.dbytes = b_cands + b_ivl + 4 * b_u32 + 2 * b_u8 + b_scr + b_cnt + b_state + b_tab;
    r.dblk = static_cast<char *>(v->dev.alloc(r.dbytes));
    if (!r.dblk) return FEM_EADMIT;
    r.hbytes = b_u32 + b_u8 + 256 + b_cands + b_ivl;
    r.hblk = static_cast<char *>(v->host.alloc(r.hbytes));
    if (!r.hblk) {
        v->dev.release(r.dblk, r.dbytes);
        return FEM_EADMIT;
    }
    char *d = r.dblk;
    r.cands = reinterpret_cast<fem_episode *>(d), d += b_cands;
    r.ivl = reinterpret_cast<uint2 *>(d), d += b_ivl;
    r.rel = reinterpret_cast<uint32_t *>(d), d += b_u32;
    r.idx = reinterpret_cast<uint32_t *>(d), d += b_u32;
    r.ex = reinterpret_cast<uint32_t *>(d), d += b_u32;
    r.out = reinterpret_cast<uint32_t *>(d), d += b_u32;
    r.flags = reinterpret_cast<uint8_t *>(d), d += b_u8;
    r.redo = reinterpret_cast<uint8_t *>(d), d += b_u8;
    r.scratch = reinterpret_cast<uint32_t *>(d), d += b_scr;
    r.cnt = reinterpret_cast<uint32_t *>(d);
    r.err = r.cnt + r.groups.size();
    d += b_cnt;
    if (b_state) r.state = reinterpret_cast<uint32_t *>(d);
    d += b_state;
    if (b_tab) r.tables = reinterpret_cast<uint4 *>(d);
    char *h = r.hblk;
    r.h_out = reinterpret_cast<uint32_t *>(h), h += b_u32;
    r.h_flags = reinterpret_cast<uint8_t *>(h), h += b_u8;
    r.h_err = reinterpret_cast<uint32_t *>(h), h += 256;
    r.h_cands = reinterpret_cast<fem_episode *>(h), h += b_cands;
    fem_interval *h_ivl = reinterpret_cast<fem_interval *>(h);
    for (uint32_t pos = 0; pos < m; ++pos) r.h_cands[pos] = cands[order[pos]];
    if (nI) std::memcpy(h_ivl, I, nI * sizeof(fem_interval));

    cudaSetDevice(v->device);
    r.lane = v->lanes[v->next_lane++ % v->lanes.size()];
    cudaStream_t st = r.lane;
    auto fail = [&](int rc) {
        cudaStreamSynchronize(st);
        v->dev.release(r.dblk, r.dbytes);
        v->host.release(r.hblk, r.hbytes);
        return rc;
    };
    if (cudaStreamWaitEvent(st, ss.ingested, 0) != cudaSuccess ||
        cudaMemcpyAsync(r.cands, r.h_cands, (size_t)m * 16, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        (nI && cudaMemcpyAsync(r.ivl, h_ivl, nI * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
        cudaMemsetAsync(r.err, 0, 4, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(FEM_ECUDA);
    }
    if (s.t_max > kServeMaxTime) return fail(FEM_ERANGE);
    if (mode == FEM_REQ_ONESHOT) {
        int rc = enqueue_oneshot(v, r, s, 0);
        if (rc == FEM_OK) rc = finish_enqueue(v, r, ss);
        if (rc != FEM_OK) return fail(rc);
    } else {
        r.ev_begin = r.ev_end;
        r.first_event = r.ev_end;
        if (cudaMemsetAsync(r.state, 0, state_words * 4, st) != cudaSuccess ||
            cudaMemsetAsync(r.out, 0, (size_t)m * 4, st) != cudaSuccess) {
            cudaGetLastError();
            return fail(FEM_ECUDA);
        }
        r.pub_counts.assign(m, 0);
        r.pub_begin = r.pub_end = r.ev_end;
        r.fresh = true;
    }
    r.holds_slot = true;
    v->active++;
    v->next_req++;
    *req_out = r.id;
    v->reqs[r.id] = std::move(r);
    return FEM_OK;
}

int fem_server_poll(fem_server *v, uint64_t *done_ids, uint32_t cap, uint32_t *n_done) {
    if (!v || (cap && !done_ids)) return FEM_EINVAL;
    cudaSetDevice(v->device);
    reap_staging(v, false);
    // retire finished work
    for (auto &kv : v->reqs) {
        Request &r = kv.second;
        if (!r.in_flight) continue;
        const cudaError_t q = cudaEventQuery(r.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) {
            cudaGetLastError();
            r.status = FEM_ECUDA;
        }
        r.in_flight = false;
        const uint32_t e = *r.h_err;
        if (e & ERR_TIMEOUT) r.status = FEM_ETIMEOUT;
        else if (e & ERR_BADEP) r.status = FEM_EINVAL;
        else if ((e & (ERR_RING | ERR_CLASS | ERR_TABLE)) && r.mode == FEM_REQ_ONESHOT &&
                 r.status == FEM_OK) {
            // a capacity guard tripped: recount with more entry classes per table, then
            // in one segment with larger rings, synchronously on the request's lane
            auto sit = v->streams.find(r.sid);
            int rc = FEM_OK;
            bool still = true;
            for (int attempt = 1; attempt <= 2 && still && rc == FEM_OK; ++attempt) {
                rc = cudaMemsetAsync(r.err, 0, 4, r.lane) == cudaSuccess ? FEM_OK : FEM_ECUDA;
                if (rc == FEM_OK) rc = enqueue_oneshot(v, r, sit->second.s, attempt);
                if (rc == FEM_OK) rc = finish_enqueue(v, r, sit->second);
                if (rc == FEM_OK && cudaEventSynchronize(r.done) != cudaSuccess) rc = FEM_ECUDA;
                still = (*r.h_err & (ERR_RING | ERR_CLASS | ERR_TABLE)) != 0;
            }
            r.in_flight = false;
            if (rc != FEM_OK) r.status = rc;
            else if (still) r.status = FEM_EOVERFLOW;
        } else if (e & ERR_RING) {
            r.status = FEM_EOVERFLOW;  // a standing request's carried lists overflowed
        }
        r.pub_counts.assign(r.h_out, r.h_out + r.m);
        if (r.mode == FEM_REQ_ONESHOT) r.pub_flags.assign(r.h_flags, r.h_flags + r.m);
        r.pub_begin = r.mode == FEM_REQ_ONESHOT ? r.ev_begin : r.first_event;
        r.pub_end = r.ev_end;
        r.fresh = true;
        if (r.mode == FEM_REQ_ONESHOT) {
            release_memory(v, r);  // results are on the host: free the slot for others
            if (r.holds_slot) {
                r.holds_slot = false;
                v->active--;
            }
        }
    }
    // advance standing requests over newly arrived events
    for (auto &kv : v->reqs) {
        Request &r = kv.second;
        if (r.mode != FEM_REQ_STANDING || r.in_flight || r.status != FEM_OK || !r.dblk) continue;
        ServeStream &ss = v->streams[r.sid];
        if (ss.s.n <= r.ev_end) continue;
        if (ss.s.t_max > kServeMaxTime) {
            r.status = FEM_ERANGE;
            continue;
        }
        r.ev_begin = r.ev_end;
        r.ev_end = ss.s.n;
        int rc = cudaStreamWaitEvent(r.lane, ss.ingested, 0) == cudaSuccess &&
                         cudaMemsetAsync(r.err, 0, 4, r.lane) == cudaSuccess
                     ? FEM_OK
                     : FEM_ECUDA;
        if (rc == FEM_OK) rc = enqueue_standing(v, r, ss.s);
        if (rc == FEM_OK) rc = finish_enqueue(v, r, ss);
        if (rc != FEM_OK) r.status = rc;
    }
    uint32_t k = 0;
    for (auto &kv : v->reqs) {
        if (!kv.second.fresh) continue;
        if (k < cap) {
            done_ids[k++] = kv.first;
            kv.second.fresh = false;
        }
    }
    if (n_done) *n_done = k;
    return FEM_OK;
}

int fem_server_result(fem_server *v, uint64_t id, uint32_t *counts_out, uint8_t *flags_out,
                      uint64_t *events_out) {
    if (!v) return FEM_EINVAL;
    auto it = v->reqs.find(id);
    if (it == v->reqs.end()) return FEM_EINVAL;
    const Request &r = it->second;
    if (r.pub_counts.size() != r.m) return FEM_EADMIT;  // no finished result yet
    for (uint32_t c = 0; c < r.m; ++c) {
        const uint32_t pos = r.perm[c];
        if (counts_out) counts_out[c] = r.pub_counts[pos];
        if (flags_out)
            flags_out[c] = r.mode == FEM_REQ_ONESHOT ? r.pub_flags[pos]
                                                     : (uint8_t)(r.pub_counts[pos] >= r.theta);
    }
    if (events_out) *events_out = r.pub_end - r.pub_begin;
    return r.status;
}

int fem_server_release(fem_server *v, uint64_t id) {
    if (!v) return FEM_EINVAL;
    auto it = v->reqs.find(id);
    if (it == v->reqs.end()) return FEM_EINVAL;
    Request &r = it->second;
    cudaSetDevice(v->device);
    if (r.in_flight) cudaEventSynchronize(r.done);
    release_memory(v, r);
    if (r.hblk) v->host.release(r.hblk, r.hbytes);
    if (r.done) v->event_pool.push_back(r.done);
    if (r.holds_slot) v->active--;
    v->reqs.erase(it);
    return FEM_OK;
}

int fem_server_drain(fem_server *v) {
    if (!v) return FEM_EINVAL;
    cudaSetDevice(v->device);
    // finish in-flight work, then let standing requests catch up with the stream
    for (int round = 0; round < 4; ++round) {
        for (cudaStream_t s : v->lanes)
            if (cudaStreamSynchronize(s) != cudaSuccess) return FEM_ECUDA;
        if (cudaStreamSynchronize(v->ingest) != cudaSuccess) return FEM_ECUDA;
        uint32_t n = 0;
        const int rc = fem_server_poll(v, nullptr, 0, &n);
        if (rc != FEM_OK) return rc;
        bool busy = false;
        for (auto &kv : v->reqs) busy |= kv.second.in_flight;
        if (!busy) return FEM_OK;
    }
    return FEM_OK;
}

}  // extern "C"
