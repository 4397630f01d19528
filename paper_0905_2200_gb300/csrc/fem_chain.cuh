// fem_chain.cuh -- the counting kernels in latest-chain form, for candidate sets whose
// episodes share prefixes (level-wise mining's candidates, any level-2 set).
//
// Both passes reduce to one rule.  For a distinct-type episode E_0 .. E_{N-1} with edge
// intervals (lo_k, hi_k], call an event i of type E_k "admitted" when it can extend some
// chain: node 0 admits every E_0 event (its chain start S(i) = i); node k > 0 admits i
// when P(i), the latest admitted E_{k-1} event strictly before i (relaxed pass,
// Algorithm 3, whose single slot holds exactly that event) or the latest one with
// t < t_i - lo_{k-1} (exact pass, Algorithm 1: the newest list entry older than lo),
// satisfies t_i - t_{P(i)} <= hi_{k-1}; then S(i) = S(P(i)).  S does not decrease along
// the admitted events of a node, so after a completion at index r the machine of
// either algorithm, whose lists were cleared, admits exactly the admitted events with
// S > r.  The count is therefore the greedy over admitted last-node events: count i
// when S(i) >= st (st = last completion + 1), then st = i + 1.  The admitted events of
// a node and their starts depend only on the episode's prefix up to that node, so the
// candidates of a block that share a prefix share its lists:
//   * per chunk, the block builds the admitted list of every distinct prefix ("node")
//     of its candidates, depth by depth (a warp per node; lists of depth-1 nodes are
//     the type groups of the staged chunk), with a bitmask over the chunk's positions
//     and per-word prefix counts, so "the latest entry before position p" is two
//     shared-memory reads and a popc; a node carries its last CH_TAIL entries into the
//     next chunk;
//   * each thread then walks only its last node's type group, looks each event up in
//     its prefix's list and applies the greedy.
// Nothing merges N type groups per thread, which is where the per-thread machine
// (fem_count.cuh) spends its instructions.  MapConcatenate (template flag MC) keeps the
// entry classes of the per-thread machine: class "none" takes chains whose first event
// is at or after the window start X (entries carry their start time), class r the
// chains after r; the transfer tables are the per-thread kernel's, so the same stitch
// composes them.  A block whose prefixes do not fit its node tables, a list longer than
// CH_LIST in one chunk, or an exact look-up that runs past a full carried tail marks
// its candidates for the host's recount (ERR_NODES; more entry classes than the thread
// tracks: ERR_CLASS), which uses the per-thread kernels.
#pragma once

#include "fem_count.cuh"

namespace fem {

constexpr int CHW = CHUNK / 32;   // bitmask words per chunk
constexpr int CH_TAIL = 8;        // entries a node carries into the next chunk
constexpr int CH_LIST = 40;       // admitted entries per node and chunk (depth >= 2)
// MapConcatenate entry classes a thread tracks (the table slots it uses), and the blocks
// per SM its register budget is set for: two-node episodes fit four blocks per SM in
// shared memory and keep four classes; longer ones fit three and keep eight.
template <int N>
constexpr int chain_classes = N == 2 ? 4 : 8;
template <int N>
constexpr int chain_blocks_per_sm = N == 2 ? 4 : 3;
// leaf events looked up per step (independent look-ups in flight; the greedy that
// consumes them stays in order): four measured slower than two at three nodes (the
// MapConcatenate form then spills: level-3 relaxed 0.46 -> 0.50 ms)
template <int N>
constexpr int chain_leaf_step = 2;

// A node's carried tail is double-buffered: lookups of chunk c read tail[c & 1] while
// the node's build for chunk c writes tail[(c + 1) & 1], so the carry needs no barrier.
struct ChainNode {
    uint32_t type, lo, hi, parent, depth, base, tlen[2];
};

// The dynamic shared memory of a chain block (named at namespace scope, so that every
// access through it is a shared-memory access with 32-bit addresses).
extern __shared__ __align__(128) uint8_t fem_chain_smem[];

template <int N, bool MC>
struct ChainLayout {
    static constexpr int NMX = N == 2 ? 16 : 34;   // nodes per block
    static constexpr int LMX = N == 2 ? 1 : 28;    // nodes of depth >= 2 (own lists)
    static constexpr int EW = MC ? 3 : 2;          // words per entry: t, S (, start time)
    static constexpr size_t META = 0;
    static constexpr size_t BITS = META + (size_t)NMX * sizeof(ChainNode);
    static constexpr size_t PRE = BITS + (size_t)NMX * CHW * 4;
    static constexpr size_t TAIL = PRE + (size_t)NMX * CHW * 2;
    static constexpr size_t LIST = TAIL + (size_t)2 * NMX * EW * CH_TAIL * 4;
    static constexpr size_t KEYS = LIST + (size_t)LMX * EW * CH_LIST * 4;
    // per-thread rows [q][T]: the part flags (row 0) and the class keys (rows 1..)
    static size_t bytes(uint32_t T) { return KEYS + (size_t)(MC ? chain_classes<N> : 1) * T * 4; }
};

// Block-wide exclusive scan of one value per thread (blockDim.x a multiple of 32, <= 1024).
__device__ __forceinline__ uint32_t chain_block_scan(uint32_t v, uint32_t *total, uint32_t *ws) {
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= (uint32_t)d) inc += y;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (uint32_t k = 0; k < nw; ++k) {
        const uint32_t x = ws[k];
        if (k < w) before += x;
        all += x;
    }
    __syncthreads();
    *total = all;
    return before + inc - v;
}

template <int N, int PASS, bool MC>
struct ChainBlock {
    using LY = ChainLayout<N, MC>;
    static constexpr int EW = LY::EW;
    // byte offsets in the block's shared memory: the node tables (nb) and the staged
    // chunk this pass reads (evb: events grouped by type, then the group offsets)
    uint32_t nb, evb;
    uint32_t n1;        // nodes of depth 1 (list slots start after them)
    uint32_t cbase;
    uint32_t par;       // tail buffer the lookups of this chunk read

    __device__ __forceinline__ ChainNode *meta() const {
        return reinterpret_cast<ChainNode *>(fem_chain_smem + nb + LY::META);
    }
    __device__ __forceinline__ uint32_t *bits() const {  // [NMX][CHW]
        return reinterpret_cast<uint32_t *>(fem_chain_smem + nb + LY::BITS);
    }
    __device__ __forceinline__ uint16_t *pre() const {  // [NMX][CHW]
        return reinterpret_cast<uint16_t *>(fem_chain_smem + nb + LY::PRE);
    }
    __device__ __forceinline__ uint32_t *tail() const {  // [2][NMX][EW][CH_TAIL]
        return reinterpret_cast<uint32_t *>(fem_chain_smem + nb + LY::TAIL);
    }
    __device__ __forceinline__ uint32_t *list() const {  // [LMX][EW][CH_LIST]
        return reinterpret_cast<uint32_t *>(fem_chain_smem + nb + LY::LIST);
    }
    __device__ __forceinline__ const uint2 *ev() const {
        return reinterpret_cast<const uint2 *>(fem_chain_smem + evb);
    }
    __device__ __forceinline__ const uint16_t *off() const {
        return reinterpret_cast<const uint16_t *>(fem_chain_smem + evb + CHUNK * 8u);
    }

    __device__ __forceinline__ uint32_t *tail_of(uint32_t nd, uint32_t which) const {
        return tail() + (which * LY::NMX + nd) * EW * CH_TAIL;
    }

    // Entry idx of node nd: idx in [-tlen, len), negative indices in the carried tail.
    // D1: the node has depth 1 (its list is its type group in the staged chunk).
    template <bool D1>
    __device__ __forceinline__ void entry(uint32_t nd, uint32_t tlen, uint32_t base, int idx,
                                          uint32_t &t, uint32_t &S, uint32_t &St) const {
        if (idx < 0) {
            const uint32_t *tp = tail_of(nd, par) + (uint32_t)((int)tlen + idx);
            t = tp[0];
            S = tp[CH_TAIL];
            St = MC ? tp[2 * CH_TAIL] : 0u;
        } else if (D1) {
            const uint2 e = ev()[base + (uint32_t)idx];
            t = e.x;
            S = cbase + e.y;
            St = e.x;
        } else {
            const uint32_t *lp = list() + (nd - n1) * EW * CH_LIST + (uint32_t)idx;
            t = lp[0];
            S = lp[CH_LIST];
            St = MC ? lp[2 * CH_LIST] : 0u;
        }
    }

    // Latest entry of node nd before chunk position pos (relaxed) or, exact, the latest
    // with t < ti - lo.  False if there is none; ovf when an exact walk ran past a full
    // carried tail (an older entry may have been dropped).
    template <bool D1>
    __device__ __forceinline__ bool lookup(uint32_t nd, uint32_t tlen, uint32_t base, uint32_t pos,
                                           uint32_t ti, uint32_t lo, uint32_t &t, uint32_t &S,
                                           uint32_t &St, bool &ovf) const {
        const uint32_t w = pos >> 5;
        int idx = (int)pre()[nd * CHW + w] + __popc(bits()[nd * CHW + w] & ((1u << (pos & 31)) - 1u)) - 1;
        const int tl = (int)tlen;
        for (;;) {
            if (idx < -tl) {
                if (PASS == FEM_PASS_EXACT && tl == CH_TAIL) ovf = true;
                return false;
            }
            entry<D1>(nd, tlen, base, idx, t, S, St);
            if (PASS == FEM_PASS_RELAXED || ti - t > lo) return true;
            --idx;
        }
    }

    // per-word prefix counts of node nd's bitmask (one warp)
    __device__ __forceinline__ void prefix(uint32_t nd, uint32_t lane) const {
        const uint32_t a = __popc(bits()[nd * CHW + 2 * lane]);
        const uint32_t b = __popc(bits()[nd * CHW + 2 * lane + 1]);
        uint32_t inc = a + b;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= (uint32_t)d) inc += y;
        }
        const uint32_t ex = inc - a - b;
        pre()[nd * CHW + 2 * lane] = (uint16_t)ex;
        pre()[nd * CHW + 2 * lane + 1] = (uint16_t)(ex + a);
    }

    // This chunk's admitted list of node nd (one warp), then the node's tail for the next
    // chunk; returns true on list overflow.
    __device__ __forceinline__ bool build(uint32_t nd, uint32_t lane) const {
        ChainNode &n = meta()[nd];
        const uint32_t g0 = off()[n.type], g1 = off()[n.type + 1];
        bits()[nd * CHW + lane] = 0;
        bits()[nd * CHW + lane + 32] = 0;
        __syncwarp();
        bool ovf = false;
        uint32_t len;
        if (n.depth == 1) {
            for (uint32_t j = g0 + lane; j < g1; j += 32) {
                const uint32_t pos = ev()[j].y;
                atomicOr(&bits()[nd * CHW + (pos >> 5)], 1u << (pos & 31));
            }
            len = g1 - g0;
            if (lane == 0) n.base = g0;
        } else {
            const uint32_t pn = n.parent, lo = n.lo, hi = n.hi;
            const uint32_t ptl = meta()[pn].tlen[par], pbase = meta()[pn].base;
            const bool pd1 = meta()[pn].depth == 1;
            uint32_t *lp = list() + (nd - n1) * EW * CH_LIST;
            uint32_t cnt = 0;
            for (uint32_t j0 = g0; j0 < g1; j0 += 32) {
                const uint32_t j = j0 + lane;
                bool adm = false;
                uint32_t ti = 0, pos = 0, t = 0, S = 0, St = 0;
                if (j < g1) {
                    const uint2 e = ev()[j];
                    ti = e.x, pos = e.y;
                    adm = (pd1 ? lookup<true>(pn, ptl, pbase, pos, ti, lo, t, S, St, ovf)
                               : lookup<false>(pn, ptl, pbase, pos, ti, lo, t, S, St, ovf)) &&
                          ti - t <= hi;
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, adm);
                const uint32_t k = cnt + __popc(bal & ((1u << lane) - 1u));
                if (adm) {
                    if (k < (uint32_t)CH_LIST) {
                        lp[k] = ti;
                        lp[CH_LIST + k] = S;
                        if (MC) lp[2 * CH_LIST + k] = St;
                        atomicOr(&bits()[nd * CHW + (pos >> 5)], 1u << (pos & 31));
                    } else {
                        ovf = true;
                    }
                }
                cnt += __popc(bal);
            }
            len = min(cnt, (uint32_t)CH_LIST);
        }
        __syncwarp();
        prefix(nd, lane);
        // the next chunk's tail: the last CH_TAIL entries of this tail followed by the list
        const uint32_t tl = n.tlen[par];
        const uint32_t nl = min((uint32_t)CH_TAIL, tl + len);
        if (lane < nl) {  // index into [-tl, len)
            uint32_t t = 0, S = 0, St = 0;
            if (n.depth == 1) entry<true>(nd, tl, g0, (int)(len - nl + lane), t, S, St);
            else entry<false>(nd, tl, g0, (int)(len - nl + lane), t, S, St);
            uint32_t *tp = tail_of(nd, par ^ 1u) + lane;
            tp[0] = t;
            tp[CH_TAIL] = S;
            if (MC) tp[2 * CH_TAIL] = St;
        }
        if (lane == 0) n.tlen[par ^ 1u] = nl;
        __syncwarp();
        return __any_sync(0xffffffffu, ovf);
    }
};

// Count one (tile of candidates, segment) in latest-chain form.  A tile whose prefixes
// do not fit the node tables is counted in parts, each over the candidates of a run of
// its leaf-parent prefixes (the segment's chunks are streamed once per part).
template <int N, int PASS, bool MC>
__device__ __forceinline__ void chain_block(const CountParams &p) {
    static_assert(N >= 2, "one-node episodes are counted by the per-thread kernels");
    using LY = ChainLayout<N, MC>;
    // entry classes tracked per thread (a window holding more capable last-node events
    // sends the episode to the recount, whose tables have S_RECOUNT slots)
    constexpr int SC = MC ? chain_classes<N> : 1;
    // leaf-parent prefixes per part when a tile must be split (their ancestors are few in
    // canonical order; a part that still overflows goes to the recount)
    constexpr uint32_t PCAP = N == 2 ? (uint32_t)LY::NMX : (uint32_t)LY::LMX;
    uint8_t *smem = fem_chain_smem;
    const uint32_t SB = stage_bytes(p.offs);
    const uint32_t T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nwarps = T >> 5;
    uint64_t *bar = stage_bars(smem, SB);
    uint32_t *sc = reinterpret_cast<uint32_t *>(smem + 2 * SB + 16);  // scalars (27 words)
    // sc[0] first chunk, sc[1] bad, sc[2..9] node base per depth, sc[10..17] nodes per depth,
    // sc[18..25] scan scratch (one word per warp is enough for 8 warps; 256 threads max)
    uint8_t *nodes = smem + 2 * SB + 128;
    ChainBlock<N, PASS, MC> cb;
    cb.nb = 2 * SB + 128;
    cb.evb = 0;
    // per-thread rows [q][T]: row 0 the part flags, rows 1.. the class keys
    uint32_t *keys_s = reinterpret_cast<uint32_t *>(nodes + LY::KEYS) + tid;

    init_stage_bars(smem, SB);
    const uint32_t m_cur = p.m_dev ? *p.m_dev : p.m;
    const uint32_t tile = blockIdx.x, seg = blockIdx.y;
    if (tile * T >= m_cur) return;  // uniform
    const uint32_t ci = tile * T + tid;

    // ------------------------------------------------------------ candidate
    uint4 rec = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
    bool ok = false;
    uint32_t E[N], lo_[N - 1], hi_[N - 1];
    if (ci < m_cur) {
        rec = reinterpret_cast<const uint4 *>(p.cands)[p.gather ? p.gather[ci] : ci];
        const uint8_t *b = reinterpret_cast<const uint8_t *>(&rec);
        ok = b[15] == N;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            E[k] = b[k];
            ok = ok && E[k] < p.K;
        }
#pragma unroll
        for (int k = 0; k < N - 1; ++k) {
            const uint32_t iv = b[8 + k];
            ok = ok && iv < p.n_ivl;
            const uint2 q = p.ivl[iv < p.n_ivl ? iv : 0];
            lo_[k] = q.x, hi_[k] = q.y;
        }
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int c = a + 1; c < N; ++c) ok = ok && E[a] != E[c];
        if (!ok) atomicOr(p.err, ERR_BADEP);
        if (!ok) rec = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) E[k] = 0;
#pragma unroll
        for (int k = 0; k < N - 1; ++k) lo_[k] = hi_[k] = 0;
    }
    // which prefix depths this candidate shares with the previous thread's (the stage
    // buffer is free until the first copy is issued)
    uint32_t same_mask = 0;
    {
        uint4 *recs = reinterpret_cast<uint4 *>(smem);
        recs[tid] = rec;
        __syncthreads();
        const uint4 prev = tid > 0 ? recs[tid - 1] : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu,
                                                                  0xFFFFFFFFu, 0xFFFFFFFFu);
        const uint64_t ta = ((uint64_t)rec.y << 32) | rec.x, tb = ((uint64_t)prev.y << 32) | prev.x;
        const uint64_t ia = ((uint64_t)rec.w << 32) | rec.z, ib = ((uint64_t)prev.w << 32) | prev.z;
#pragma unroll
        for (int d = 1; d <= N - 1; ++d) {
            const uint64_t tm = d >= 8 ? ~0ull : ((1ull << (8 * d)) - 1ull);
            const uint64_t im = (d - 1) >= 8 ? ~0ull : ((1ull << (8 * (d - 1))) - 1ull);
            if (((ta ^ tb) & tm) == 0 && ((ia ^ ib) & im) == 0) same_mask |= 1u << d;
        }
    }
    // parts: the whole tile if its prefixes fit the tables, else runs of PCAP
    // leaf-parent prefixes
    uint32_t lp_rank = 0, lp_total = 0;
    {
        const uint32_t is_new = ok && !((same_mask >> (N - 1)) & 1u);
        const uint32_t ex = chain_block_scan(is_new, &lp_total, sc + 18);
        lp_rank = ex + is_new - 1u;  // ok threads
    }
    bool split = false;
    uint32_t part = 0, nparts = 1;

    // ------------------------------------------------------------ segment and window
    const uint32_t c_seg0 = seg * p.cps;
    const uint32_t c_end = min(c_seg0 + p.cps, p.n_chunks);
    const uint32_t L = c_seg0 * CHUNK;
    uint32_t X = 0, Xn = 0, c_w = c_seg0;
    const bool last_seg = c_end >= p.n_chunks;
    if (MC) {
        uint64_t W = 0;
#pragma unroll
        for (int k = 0; k < N - 1; ++k) W += hi_[k];
        if (ok && seg > 0) {
            const uint32_t tL = p.cfirst[c_seg0];
            X = (uint64_t)tL >= W ? (uint32_t)(tL - W) : 0u;
            const uint32_t X2 = (uint64_t)tL >= 2 * W ? (uint32_t)(tL - 2 * W) : 0u;
            uint32_t c = c_seg0;
            if (X2 == 0) c = 0;
            else
                while (c > 0 && p.cfirst[c] >= X2) --c;
            c_w = c;
        }
        if (!last_seg) {
            const uint32_t tR = p.cfirst[c_end];
            Xn = (uint64_t)tR >= W ? (uint32_t)(tR - W) : 0u;
        }
    }
    const uint32_t El = E[N - 1], lo = lo_[N - 2], hi = hi_[N - 2];
    const uint32_t chunk_ev_bytes = CHUNK * 8u;
    const uint32_t chunk_off_bytes = p.offs * 2u;
    auto issue = [&](uint32_t c, uint32_t s) {
        uint8_t *dst = smem + s * SB;
        mbar_expect_tx(&bar[s], chunk_ev_bytes + chunk_off_bytes);
        bulk_g2s(dst, p.bev + (uint64_t)c * CHUNK, chunk_ev_bytes, &bar[s]);
        bulk_g2s(dst + chunk_ev_bytes, p.boff + (uint64_t)c * p.offs, chunk_off_bytes, &bar[s]);
    };
    uint32_t jbase = 0;  // chunk stages consumed so far (their mbarrier phases)

    for (uint32_t pt = 0; pt < nparts; ++pt) {
        const bool act = ok && (!split || part == pt);
        // ------------------------------------------------------------ this part's nodes
        // node of each depth d (1..N-1): the prefix E_0..E_{d-1} with its d-1 edges; an
        // active thread opens a node where its prefix differs from the previous thread's
        // or the previous thread is not in this part
        keys_s[0] = act;
        __syncthreads();
        const bool prev_act = tid > 0 && keys_s[-1] != 0;
        uint32_t nid[N];
        uint32_t n_total = 0, n1 = 0;
#pragma unroll
        for (int d = 1; d <= N - 1; ++d) {
            const uint32_t is_new = act && !(prev_act && ((same_mask >> d) & 1u));
            uint32_t tot;
            const uint32_t ex = chain_block_scan(is_new, &tot, sc + 18);
            nid[d] = n_total + ex + is_new - 1u;  // active threads: the latest node opened
            if (tid == 0) sc[2 + d] = n_total, sc[10 + d] = tot;
            if (is_new && n_total + ex < (uint32_t)LY::NMX) {
                ChainNode *nd = cb.meta() + n_total + ex;
                nd->type = E[d - 1];
                nd->lo = d >= 2 ? lo_[d - 2] : 0u;
                nd->hi = d >= 2 ? hi_[d - 2] : 0u;
                nd->parent = d >= 2 ? nid[d - 1] : 0u;
                nd->depth = (uint32_t)d;
                nd->base = 0, nd->tlen[0] = 0, nd->tlen[1] = 0;
            }
            if (d == 1) n1 = tot;
            n_total += tot;
        }
        if (tid == 0) sc[0] = c_seg0, sc[1] = 0;
        __syncthreads();  // node records, counts and the scalars are visible
        cb.n1 = n1;
        if (n_total > (uint32_t)LY::NMX || n_total - n1 > (uint32_t)LY::LMX) {
            // the whole tile does not fit: count it in parts (uniform); two-node tiles in
            // canonical order have a few first types, so they go to the recount instead
            if (N >= 3 && !split) {
                split = true;
                part = lp_rank / PCAP;
                nparts = (lp_total + PCAP - 1) / PCAP;
                pt = ~0u;  // the loop's increment starts the parts at 0
                continue;
            }
            // even this part's prefixes do not fit: its candidates go to the host's recount
            if (act) p.redo[ci] = 1;
            if (tid == 0) atomicOr(p.err, ERR_NODES);
            continue;  // uniform
        }
        const uint32_t pn = nid[N - 1];  // the leaf's parent node
        if (MC && act) atomicMin(&sc[0], c_w);
        __syncthreads();
        const uint32_t c_first = MC ? sc[0] : c_seg0;

        // ------------------------------------------------------------ counting state
        // single segment: st = last completion + 1.  MapConcatenate: per entry class its
        // st, count and (class "none" aside) key, as in the per-thread kernel
        uint32_t cnt = 0, st = 0;
        uint32_t c_st[SC], c_cnt[SC];
#pragma unroll
        for (int j = 0; j < SC; ++j) c_st[j] = 0, c_cnt[j] = 0;
        uint32_t used = 0, umask = 0;
        bool c0_done = false, class_overflow = false, ovf = false;
        auto set_key = [&](int q0, uint32_t v) { keys_s[(uint32_t)q0 * T] = v; };
        auto get_key = [&](int q) -> uint32_t { return q == 0 ? CLS_NONE : keys_s[(uint32_t)q * T]; };

        // ------------------------------------------------------------ chunk pipeline
        if (tid == 0) {
            fence_proxy_async_smem();
            if (c_first < c_end) issue(c_first, jbase & 1u);
            if (c_first + 1 < c_end) issue(c_first + 1, (jbase + 1) & 1u);
        }
        bool bail = false;
        uint32_t c = c_first;
        for (; c < c_end; ++c) {
            const uint32_t j = jbase + (c - c_first), s = j & 1u, par = (j >> 1) & 1u;
            const bool waited = mbar_wait_bounded(&bar[s], par, p.err);
            if (!__syncthreads_and(waited)) {
                bail = true;
                break;
            }
            cb.evb = s * SB;
            cb.cbase = c * CHUNK;
            cb.par = (c - c_first) & 1u;
            // prefix lists, depth by depth (each build also writes the node's next tail)
            bool bovf = false;
            for (int d = 1; d <= N - 1; ++d) {
                const uint32_t b0 = sc[2 + d], nb = sc[10 + d];
                for (uint32_t nd = b0 + warp; nd < b0 + nb; nd += nwarps) bovf |= cb.build(nd, lane);
                __syncthreads();
            }
            if (bovf && lane == 0) sc[1] = 1;
            // the leaf: this thread's last node's events, looked up in the parent's list
            if (act && c >= c_w) {
                const uint32_t g0 = cb.off()[El], g1 = cb.off()[El + 1];
                const uint32_t ptl = cb.meta()[pn].tlen[cb.par], pbase = cb.meta()[pn].base;
                auto adm_at = [&](const uint2 e, uint32_t &S, uint32_t &St) -> bool {
                    uint32_t t;
                    return cb.template lookup<N == 2>(pn, ptl, pbase, e.y, e.x, lo, t, S, St, ovf) &&
                           e.x - t <= hi;
                };
                if (!MC || (c >= c_seg0 && umask == 0)) {
                    // one class: inside the segment with every entry class merged, or one
                    // segment.  Several events per step: their look-ups are independent,
                    // the greedy is not.
                    auto apply = [&](bool a, uint32_t y, uint32_t S, uint32_t St) {
                        if (!a) return;
                        const uint32_t gidx = cb.cbase + y;
                        if constexpr (!MC) {
                            if (S >= st) ++cnt, st = gidx + 1;
                        } else {
                            if (S >= c_st[0] && St >= X) c_st[0] = gidx + 1, ++c_cnt[0], c0_done = true;
                        }
                    };
                    constexpr int U = chain_leaf_step<N>;
                    uint32_t jj = g0;
                    for (; jj + U <= g1; jj += U) {
                        uint2 e[U];
                        uint32_t S[U], St[U];
                        bool a[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) e[u] = cb.ev()[jj + u];
#pragma unroll
                        for (int u = 0; u < U; ++u) a[u] = adm_at(e[u], S[u], St[u]);
#pragma unroll
                        for (int u = 0; u < U; ++u) apply(a[u], e[u].y, S[u], St[u]);
                    }
                    for (; jj < g1; ++jj) {
                        const uint2 e = cb.ev()[jj];
                        uint32_t S, St;
                        const bool a = adm_at(e, S, St);
                        apply(a, e.y, S, St);
                    }
                } else if constexpr (MC) {
                    for (uint32_t jj = g0; jj < g1; ++jj) {
                        const uint2 e = cb.ev()[jj];
                        uint32_t S, St, tp;
                        const bool found = cb.template lookup<N == 2>(pn, ptl, pbase, e.y, e.x, lo,
                                                                       tp, S, St, ovf);
                        if (!found) continue;
                        // Every later event of this node looks up this parent entry or a
                        // later one, so its chain starts at S or later: a class whose
                        // threshold is at most S admits all of them, as class "none" does
                        // when its conditions hold for S too -- such a class behaves like
                        // class "none" from here on.
                        if (umask && S >= c_st[0] && St >= X) {
#pragma unroll
                            for (int q = 1; q < SC; ++q) {
                                if (((umask >> q) & 1u) && c_st[q] <= S) {
                                    c_cnt[q] -= c_cnt[0];
                                    umask &= ~(1u << q);
                                    if (cb.cbase + e.y < L) used &= ~(1u << q);
                                }
                            }
                        }
                        if (e.x - tp > hi) continue;
                        const uint32_t ti = e.x, gidx = cb.cbase + e.y;
                        const uint32_t inc = gidx >= L ? 1u : 0u;
                        if (S >= c_st[0] && St >= X) c_st[0] = gidx + 1, c_cnt[0] += inc, c0_done = true;
                        if (umask) {
#pragma unroll
                            for (int q = 1; q < SC; ++q) {
                                if (!((umask >> q) & 1u)) continue;
                                if (S >= c_st[q]) {
                                    if (!inc) {  // refuted: completes before the segment
                                        used &= ~(1u << q), umask &= ~(1u << q);
                                        continue;
                                    }
                                    c_st[q] = gidx + 1, ++c_cnt[q];
                                }
                                if (c_st[q] == c_st[0]) {
                                    c_cnt[q] -= c_cnt[0];
                                    umask &= ~(1u << q);
                                    if (!inc) used &= ~(1u << q);
                                }
                            }
                        }
                        if (!inc && ti >= X && c_st[0] != gidx + 1) {
                            // entry class r = gidx: the chains after it
                            constexpr uint32_t all_slots = SC >= 32 ? 0xFFFFFFFFu : (1u << SC) - 1u;
                            const uint32_t free_slots = ~used & (all_slots & ~1u);
                            if (free_slots) {
                                const int qn = __ffs(free_slots) - 1;
                                set_key(qn, gidx);
#pragma unroll
                                for (int q = 1; q < SC; ++q)
                                    if (q == qn) c_st[q] = gidx + 1, c_cnt[q] = 0;
                                used |= 1u << qn;
                                umask |= 1u << qn;
                            } else {
                                class_overflow = true;
                            }
                        }
                    }
                }
            }
            // (a barrier, not the next chunk's mbarrier wait, holds the threads that are
            // done early: their spinning would take issue slots from the others)
            __syncthreads();
            if (tid == 0 && c + 2 < c_end) {
                fence_proxy_async_smem();
                issue(c + 2, s);
            }
        }
        if (bail) {
            if (tid == 0) {
                for (uint32_t cc = c; cc < min(c + 2, c_end); ++cc) {
                    const uint32_t jq = jbase + (cc - c_first);
                    mbar_wait_bounded(&bar[jq & 1u], (jq >> 1) & 1u, p.err);
                }
            }
            return;
        }
        jbase += c_end > c_first ? c_end - c_first : 0u;

        // ------------------------------------------------------------ results
        if (ci < m_cur && !ok && !MC) p.out[ci] = 0;
        const bool mine = act || (!ok && ci < m_cur && pt + 1 == nparts);
        if (!mine) continue;
        const bool bad = act && (sc[1] != 0 || ovf || class_overflow);
        if (bad) {
            atomicOr(p.err, (class_overflow ? ERR_CLASS : 0u) | (ovf || sc[1] != 0 ? ERR_NODES : 0u));
            p.redo[ci] = 1;
        }
        if constexpr (!MC) {
            p.out[ci] = act ? cnt : 0u;
        } else {
            uint4 *tab = p.tables + ((uint64_t)seg * p.m + ci) * S_MAX;
            const uint32_t n_slots = used ? 32u - __clz(used) : 1u;
            static_assert(SC <= S_MAX, "the transfer tables hold S_MAX classes");
#pragma unroll
            for (int q = 0; q < SC; ++q) {
                if ((uint32_t)q >= n_slots) break;
                uint4 e = make_uint4(CLS_EMPTY, 0, CLS_NONE, q == 0 ? n_slots : 0u);
                if (act && (q == 0 || ((used >> q) & 1u))) {
                    const bool merged = q > 0 && !((umask >> q) & 1u);
                    const uint32_t cntq = merged ? c_cnt[0] + c_cnt[q] : c_cnt[q];
                    const uint32_t stq = merged ? c_st[0] : c_st[q];
                    uint32_t ex = (q == 0 && !c0_done) ? CLS_NONE : stq - 1u;
                    if (ex != CLS_NONE && !last_seg && p.t[ex] < Xn) ex = CLS_NONE;
                    e = make_uint4(get_key(q), cntq, ex, q == 0 ? n_slots : 0u);
                }
                tab[q] = e;
            }
        }
    }
}

template <int N, int PASS, bool MC>
__global__ void __launch_bounds__(256, chain_blocks_per_sm<N>) k_chain(const CountParams p) {
    chain_block<N, PASS, MC>(p);
}

}  // namespace fem
