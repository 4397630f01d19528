// fem_pairs.cu -- the relaxed pass (Algorithm 3) over a complete level-2 candidate set
// (fem_count_pairs_relaxed) with every interval variant of one ordered type pair counted
// by one thread.
//
// Level 2 holds, for each ordered pair (a, b) of distinct frequent types, one candidate
// per interval of I (canonical order: the candidate with interval v sits at
// a_i * nI * nb + v * nb + b_j, nb = f - 1).  For two nodes Algorithm 3 reduces to the
// latest-chain rule (fem_chain.cuh): event i of type b is admitted by the variant with
// interval hi_v when P(i), the latest a-event before it, satisfies t_i - t_P <= hi_v,
// and the variant counts i when P(i) >= st_v (st_v = its last completion + 1).  P(i) is
// the same for every variant, so a thread merges the pair's two type groups once and
// keeps per variant only its threshold, its count and, with MapConcatenate, its entry
// classes (the chain kernels' class rules: class "none" takes chains that start at or
// after the variant's window start X_v, class r the chains after r).  The transfer
// tables and output slots are the generic kernels' (indexed by the candidate), so the
// same stitch composes them and the host's recount serves flagged candidates.
#include "fem_count.cuh"

namespace fem {

constexpr int kPairVariants = 4;   // interval variants per thread (|I| <= 4)
constexpr int kPairClasses = 4;    // entry-class slots per variant

template <bool MC>
__global__ void __launch_bounds__(256, 3) k_pairs_relaxed(const CountParams p) {
    constexpr int V = kPairVariants, SC = MC ? kPairClasses : 1;
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t SB = stage_bytes(p.offs);
    const uint32_t T = blockDim.x, tid = threadIdx.x;
    uint64_t *bar = stage_bars(smem, SB);
    // class keys, [variant][slot][thread]
    uint32_t *keys = reinterpret_cast<uint32_t *>(smem + 2 * SB + 128);
    init_stage_bars(smem, SB);

    const uint32_t nI = p.n_ivl, nb = p.pair_types - 1, n_pairs = p.pair_types * nb;
    if (blockIdx.x * T >= n_pairs) return;  // uniform
    const uint32_t pair = blockIdx.x * T + tid, seg = blockIdx.y;
    const uint32_t ai = pair / max(nb, 1u), bj = pair % max(nb, 1u);

    // ---------------------------------------------------------------- the pair's variants
    bool ok = pair < n_pairs && nI >= 1 && nI <= (uint32_t)V;
    // candidate of variant v: ci0 + v nb
    const uint32_t ci0 = ai * nI * nb + bj;
    uint32_t A = 0, B = 0, hi[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        hi[v] = 0;
        if (ok && (uint32_t)v < nI) {
            const fem_episode e = p.cands[ci0 + (uint32_t)v * nb];
            if (v == 0) A = e.types[0], B = e.types[1];
            const uint32_t iv = e.ivl[0];
            ok = ok && e.len == 2 && e.types[0] == A && e.types[1] == B && iv == (uint32_t)v &&
                 A != B && A < p.K && B < p.K;
            hi[v] = p.ivl[iv < p.n_ivl ? iv : 0].y;
        }
    }
    if (pair < n_pairs && !ok) atomicOr(p.err, ERR_BADEP);

    // ---------------------------------------------------------------- segment and windows
    const uint32_t c_seg0 = seg * p.cps;
    const uint32_t c_end = min(c_seg0 + p.cps, p.n_chunks);
    const uint32_t L = c_seg0 * CHUNK;
    const bool last_seg = c_end >= p.n_chunks;
    // variant v's window starts X_v = tL - hi_v (this segment) and tR - hi_v (the next)
    uint32_t tL = 0, tR = 0, c_w = c_seg0;
    if (MC && ok) {
        uint32_t Wm = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) Wm = max(Wm, hi[v]);
        if (seg > 0) {
            tL = p.cfirst[c_seg0];
            const uint32_t X2 = (uint64_t)tL >= 2ull * Wm ? (uint32_t)(tL - 2 * Wm) : 0u;
            uint32_t c = c_seg0;
            if (X2 == 0) c = 0;
            else
                while (c > 0 && p.cfirst[c] >= X2) --c;
            c_w = c;
        }
        if (!last_seg) tR = p.cfirst[c_end];
    }
    auto X = [&](int v) { return tL >= hi[v] ? tL - hi[v] : 0u; };
    auto Xn = [&](int v) { return tR >= hi[v] ? tR - hi[v] : 0u; };
    // the block starts at its earliest window
    uint32_t *s_cw = reinterpret_cast<uint32_t *>(smem + 2 * SB + 16);
    if (tid == 0) *s_cw = c_seg0;
    __syncthreads();
    if (MC && ok) atomicMin(s_cw, c_w);
    __syncthreads();
    const uint32_t c_first = *s_cw;

    // ---------------------------------------------------------------- counting state
    uint32_t st[V][SC], cnt[V][SC];
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
        for (int q = 0; q < SC; ++q) st[v][q] = 0, cnt[v][q] = 0;
    uint32_t used[V], umask[V];
#pragma unroll
    for (int v = 0; v < V; ++v) used[v] = 0, umask[v] = 0;
    uint32_t done0 = 0, overflow = 0;  // bit per variant
    uint32_t last_t = 0, last_i = 0;   // the latest a-event seen (its time and index)
    bool have_a = false;

    // ---------------------------------------------------------------- chunk pipeline
    const uint32_t chunk_ev_bytes = CHUNK * 8u, chunk_off_bytes = p.offs * 2u;
    auto issue = [&](uint32_t c, uint32_t s) {
        uint8_t *dst = smem + s * SB;
        mbar_expect_tx(&bar[s], chunk_ev_bytes + chunk_off_bytes);
        bulk_g2s(dst, p.bev + (uint64_t)c * CHUNK, chunk_ev_bytes, &bar[s]);
        bulk_g2s(dst + chunk_ev_bytes, p.boff + (uint64_t)c * p.offs, chunk_off_bytes, &bar[s]);
    };
    if (tid == 0) {
        fence_proxy_async_smem();
        if (c_first < c_end) issue(c_first, 0);
        if (c_first + 1 < c_end) issue(c_first + 1, 1);
    }
    bool bail = false;
    uint32_t c = c_first;
    for (; c < c_end; ++c) {
        const uint32_t j = c - c_first, s = j & 1u, par = (j >> 1) & 1u;
        const bool waited = mbar_wait_bounded(&bar[s], par, p.err);
        if (!__syncthreads_and(waited)) {
            bail = true;
            break;
        }
        if (ok && c >= c_w) {
            const uint2 *ev = reinterpret_cast<const uint2 *>(smem + s * SB);
            const uint16_t *off = reinterpret_cast<const uint16_t *>(smem + s * SB + chunk_ev_bytes);
            const uint32_t cbase = c * CHUNK;
            uint32_t pa = off[A];
            const uint32_t a1 = off[A + 1], b0 = off[B], b1 = off[B + 1];
            const bool simple = !MC || c >= c_seg0;
            bool live = false;
#pragma unroll
            for (int v = 0; v < V; ++v) live = live || umask[v] != 0;
            if (simple && !live) {
                // One class per variant (one segment, or inside the segment with every
                // entry class merged).  There the window condition St >= X_v holds for
                // every admitted event: t_i >= t[L] and t_i - t_P <= hi_v.
                for (uint32_t jb = b0; jb < b1; ++jb) {
                    const uint2 eb = ev[jb];
                    while (pa < a1) {
                        const uint2 ea = ev[pa];
                        if (ea.y >= eb.y) break;
                        last_t = ea.x, last_i = cbase + ea.y, have_a = true;
                        ++pa;
                    }
                    if (!have_a) continue;
                    const uint32_t d = eb.x - last_t, nxt = cbase + eb.y + 1;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const bool cond = (uint32_t)v < nI && d <= hi[v] && last_i >= st[v][0];
                        st[v][0] = cond ? nxt : st[v][0];
                        cnt[v][0] += cond ? 1u : 0u;
                        if (MC) done0 |= (cond ? 1u : 0u) << v;
                    }
                }
                if (pa < a1) {
                    const uint2 ea = ev[a1 - 1];
                    last_t = ea.x, last_i = cbase + ea.y, have_a = true;
                }
                goto next_chunk;
            }
            for (uint32_t jb = b0; jb < b1; ++jb) {
                const uint2 eb = ev[jb];
                // the latest a-event before this b-event
                while (pa < a1) {
                    const uint2 ea = ev[pa];
                    if (ea.y >= eb.y) break;
                    last_t = ea.x, last_i = cbase + ea.y, have_a = true;
                    ++pa;
                }
                if (!have_a) continue;
                const uint32_t ti = eb.x, gidx = cbase + eb.y, S = last_i, St = last_t;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if ((uint32_t)v >= nI) continue;
                    const bool adm = ti - St <= hi[v];
                    if (!MC) {
                        if (adm && S >= st[v][0]) ++cnt[v][0], st[v][0] = gidx + 1;
                        continue;
                    }
                    if (simple && umask[v] == 0) {
                        // inside the segment with every entry class merged
                        if (adm && S >= st[v][0] && St >= X(v))
                            st[v][0] = gidx + 1, ++cnt[v][0], done0 |= 1u << v;
                        continue;
                    }
                    // Every later b-event looks up this a-event or a later one, so its
                    // chain starts at S or later: a class whose threshold is at most S
                    // behaves like class "none" from here on when "none" admits S.
                    if (umask[v] && S >= st[v][0] && St >= X(v)) {
#pragma unroll
                        for (int q = 1; q < SC; ++q) {
                            if (((umask[v] >> q) & 1u) && st[v][q] <= S) {
                                cnt[v][q] -= cnt[v][0];
                                umask[v] &= ~(1u << q);
                                if (gidx < L) used[v] &= ~(1u << q);
                            }
                        }
                    }
                    if (!adm) continue;
                    const uint32_t inc = gidx >= L ? 1u : 0u;
                    if (S >= st[v][0] && St >= X(v)) st[v][0] = gidx + 1, cnt[v][0] += inc, done0 |= 1u << v;
#pragma unroll
                    for (int q = 1; q < SC; ++q) {
                        if (!((umask[v] >> q) & 1u)) continue;
                        if (S >= st[v][q]) {
                            if (!inc) {  // refuted: completes before the segment
                                used[v] &= ~(1u << q), umask[v] &= ~(1u << q);
                                continue;
                            }
                            st[v][q] = gidx + 1, ++cnt[v][q];
                        }
                        if (st[v][q] == st[v][0]) {
                            cnt[v][q] -= cnt[v][0];
                            umask[v] &= ~(1u << q);
                            if (!inc) used[v] &= ~(1u << q);
                        }
                    }
                    if (!inc && ti >= X(v) && st[v][0] != gidx + 1) {
                        // entry class r = gidx: the chains after it
                        constexpr uint32_t all_slots = (1u << SC) - 1u;
                        const uint32_t free_slots = ~used[v] & (all_slots & ~1u);
                        if (free_slots) {
                            const int qn = __ffs(free_slots) - 1;
                            keys[((uint32_t)v * SC + (uint32_t)qn) * T + tid] = gidx;
#pragma unroll
                            for (int q = 1; q < SC; ++q)
                                if (q == qn) st[v][q] = gidx + 1, cnt[v][q] = 0;
                            used[v] |= 1u << qn;
                            umask[v] |= 1u << qn;
                        } else {
                            overflow |= 1u << v;
                        }
                    }
                }
            }
            if (pa < a1) {  // a-events after the group's last b-event
                const uint2 ea = ev[a1 - 1];
                last_t = ea.x, last_i = cbase + ea.y, have_a = true;
            }
        }
    next_chunk:
        __syncthreads();
        if (tid == 0 && c + 2 < c_end) {
            fence_proxy_async_smem();
            issue(c + 2, s);
        }
    }
    if (bail) {
        if (tid == 0) {
            for (uint32_t cc = c; cc < min(c + 2, c_end); ++cc) {
                const uint32_t jq = cc - c_first;
                mbar_wait_bounded(&bar[jq & 1u], (jq >> 1) & 1u, p.err);
            }
        }
        return;
    }

    // ---------------------------------------------------------------- results
    if (pair >= n_pairs) return;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        if ((uint32_t)v >= nI) continue;
        const uint32_t e_ci = ci0 + (uint32_t)v * nb;
        if (ok && ((overflow >> v) & 1u)) {
            atomicOr(p.err, ERR_CLASS);
            p.redo[e_ci] = 1;
        }
        if constexpr (!MC) {
            p.out[e_ci] = ok ? cnt[v][0] : 0u;
        } else {
            uint4 *tab = p.tables + ((uint64_t)seg * p.m + e_ci) * S_MAX;
            const uint32_t n_slots = used[v] ? 32u - __clz(used[v]) : 1u;
#pragma unroll
            for (int q = 0; q < SC; ++q) {
                if ((uint32_t)q >= n_slots) break;
                uint4 e = make_uint4(CLS_EMPTY, 0, CLS_NONE, q == 0 ? n_slots : 0u);
                if (ok && (q == 0 || ((used[v] >> q) & 1u))) {
                    const bool merged = q > 0 && !((umask[v] >> q) & 1u);
                    const uint32_t cq = merged ? cnt[v][0] + cnt[v][q] : cnt[v][q];
                    const uint32_t sq = merged ? st[v][0] : st[v][q];
                    uint32_t ex = (q == 0 && !((done0 >> v) & 1u)) ? CLS_NONE : sq - 1u;
                    if (ex != CLS_NONE && !last_seg && p.t[ex] < Xn(v)) ex = CLS_NONE;
                    const uint32_t key = q == 0 ? CLS_NONE : keys[((uint32_t)v * SC + (uint32_t)q) * T + tid];
                    e = make_uint4(key, cq, ex, q == 0 ? n_slots : 0u);
                }
                tab[q] = e;
            }
        }
    }
}

size_t pairs_smem_bytes(bool mc, uint32_t threads, uint32_t offs) {
    return 2 * (size_t)stage_bytes(offs) + 128 +
           (mc ? (size_t)kPairVariants * kPairClasses * threads * 4 : 0);
}

// The relaxed pass of a level-2 set of f frequent types x n_ivl intervals (m = f (f - 1)
// n_ivl candidates in canonical order, p.pair_types = f): one thread per (ordered pair,
// segment).
cudaError_t launch_pairs_relaxed(const CountParams &p, uint32_t threads, cudaStream_t st) {
    if (p.pair_types < 2 || p.n_ivl == 0 || p.n_ivl > (uint32_t)kPairVariants) return cudaErrorInvalidValue;
    if (threads < 32 || threads > 256 || threads % 32) return cudaErrorInvalidConfiguration;
    const bool mc = p.P > 1;
    const size_t sm = pairs_smem_bytes(mc, threads, p.offs);
    static bool attr_set[2] = {false, false};
    if (!attr_set[mc]) {
        const cudaError_t e = mc ? cudaFuncSetAttribute(k_pairs_relaxed<true>,
                                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        227 * 1024)
                                 : cudaFuncSetAttribute(k_pairs_relaxed<false>,
                                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        227 * 1024);
        if (e != cudaSuccess) return e;
        attr_set[mc] = true;
    }
    const uint32_t n_pairs = p.pair_types * (p.pair_types - 1);
    dim3 grid((n_pairs + threads - 1) / threads, mc ? p.P : 1);
    if (mc) k_pairs_relaxed<true><<<grid, threads, sm, st>>>(p);
    else k_pairs_relaxed<false><<<grid, threads, sm, st>>>(p);
    note_launch();
    return cudaGetLastError();
}

// Level-wise mining's use of the pass (Algorithm 4).  A candidate whose relaxed count the
// pair kernel did not finish (flagged: more entry classes than its slots, or a table the
// stitch could not compose) gets the largest count.  When such candidates are few (at
// most `limit`), that is all: they pass the elimination and the exact pass decides them
// -- the relaxed count bounds the exact one from above, so the frequent set is the same
// -- and the flags' error bits are cleared.  When they are many (bursts), the bits stay
// and the host recounts them (overwriting the largest counts) before the elimination.
// work[0..1]: zero before the launch (flag total, blocks done); the last block resets them.
__global__ void k_pairs_pass_flagged(uint32_t *__restrict__ out, const uint8_t *__restrict__ redo,
                                     uint32_t m, uint32_t limit, uint32_t *work, uint32_t *err) {
    __shared__ bool last;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool f = i < m && redo[i] != 0;
    if (f) out[i] = 0xFFFFFFFFu;
    const uint32_t nf = (uint32_t)__syncthreads_count(f);
    if (threadIdx.x == 0) {
        if (nf) atomicAdd(&work[0], nf);
        __threadfence();
        last = atomicAdd(&work[1], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const uint32_t total = atomicAdd(&work[0], 0u);
        if (total <= limit) atomicAnd(err, ~(ERR_CLASS | ERR_TABLE));
        work[0] = 0;
        work[1] = 0;
    }
}

cudaError_t launch_pairs_pass_flagged(uint32_t *out, const uint8_t *redo, uint32_t m,
                                      uint32_t limit, uint32_t *work, uint32_t *err,
                                      cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_pairs_pass_flagged<<<(m + 255) / 256, 256, 0, st>>>(out, redo, m, limit, work, err);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fem
