// fem_count.cuh -- the counting kernels (Algorithm 1 exact, Algorithm 3 relaxed),
// one thread per (episode, segment).
//
// Data flow per block: the block's threads count T episodes over one stream
// segment.  Thread 0 streams the segment's chunks into two shared-memory stages
// with 1-D bulk (TMA) copies completed on mbarriers; every thread then merges,
// by local index, the groups of its episode's N types in the staged chunk, so
// it visits exactly the events that can change its state machine, in stream
// order.  Nothing per event is read from global memory.
//
// Machines (node k = 0..N-1, edge k joins node k and k+1 with interval (lo, hi]):
//  * relaxed (Algorithm 3, Section 5.3.1): one slot per node holding the
//    deadline s + hi + 1 of the latest admitted time s (0 = unset);
//  * exact (Algorithm 1, Section 5.1): per node a FIFO ring in shared memory
//    holding the list s[k] of admitted times as clusters [first, last]: a new
//    time joins the newest cluster when it is within hi - lo of that cluster's
//    last time.  A cluster matches exactly the event times in
//    (first + lo, last + hi] (consecutive members are at most hi - lo apart, so
//    the union of their (s + lo, s + hi] ranges has no hole), which is the
//    list's own check "some t' in s[k] with lo < t - t' <= hi".  Clusters whose
//    last time is older than hi can never match again (times do not decrease)
//    and are dropped, so at most ceil(hi / (hi - lo)) clusters are live.  A ring
//    that would overflow sets ERR_RING and the host recounts the episode with a
//    larger ring.  The segmented variant keeps single times (with equal times
//    merged), because it needs the annotation of the newest matching entry.
//    When every edge has hi >= 2 lo at most two clusters are live, and the lean
//    step keeps both in registers instead of the ring.
//
// MapConcatenate (Section 5.2.2), exact form (template flag MC): the thread
// counting segment p starts at the window start w_p (first event with
// t >= t[L_p] - W, W = sum of hi) and tabulates, for each entry class
// (class "none" = no completion since before w_p, or any last-node event r in
// [w_p, L_p)), the completions inside [L_p, R_p) and the class handed to the
// next segment.  All classes are tracked by one annotated machine: every
// admitted entry carries the largest start index of a chain that reaches it,
// and a class whose machine (re)started at `start` sees exactly the entries
// whose annotation is >= start.  A completion whose annotation is ms restarts
// every class with start <= ms at the next event.  The tables are composed by
// the stitch kernel.
#pragma once

#include <type_traits>

#include "fem_internal.cuh"

namespace fem {

// Calls f(integral_constant<int, K>), f(...K-1), ..., f(...0): the node loop of
// Algorithms 1 and 3 runs from the last node down to the first.
template <int K, typename F>
__device__ __forceinline__ void for_nodes_desc(F &&f) {
    if constexpr (K >= 0) {
        f(std::integral_constant<int, K>{});
        for_nodes_desc<K - 1>(f);
    }
}

// With distinct types exactly one group's head holds the minimum key.  For two nodes
// the exact lean step tests the second group only and takes the first otherwise
// (level-2 exact 0.29 -> 0.27 ms with the same shape).  The relaxed step keeps the
// test of every group (the else-chain measured 0.29 -> 0.30 ms at level 2), and so
// do longer episodes.  With repeated types several nodes can match one event:
// for_nodes_desc.
template <int N, typename P, typename F>
__device__ __forceinline__ void lean_nodes(P &&is_min, F &&f) {
    if constexpr (N == 2) {
        if (is_min(std::integral_constant<int, 1>{})) f(std::integral_constant<int, 1>{});
        else f(std::integral_constant<int, 0>{});
    } else {
        for_nodes_desc<N - 1>([&](auto kc) {
            if (is_min(kc)) f(kc);
        });
    }
}

template <int N>
struct EpRegs {
    static constexpr int NE = N > 1 ? N - 1 : 1;
    uint32_t E[N];
    uint32_t lo[NE], hi[NE];
};

// Shared memory of a counting block: two chunk stages of SB bytes each, then two
// mbarriers and a scratch word, then the exact pass's rings.
__device__ __forceinline__ uint64_t *stage_bars(uint8_t *smem, uint32_t SB) {
    return reinterpret_cast<uint64_t *>(smem + 2 * SB);
}

// Count one work item: the block's T threads take episodes tile*T .. tile*T+T-1 of
// the candidate set over segment `seg`.  `q` is the block's running number of
// consumed chunk stages (it selects the stage and mbarrier phase of each chunk and
// carries over to the block's next item).  Returns false if a bounded wait gave up;
// the caller must then stop using the block's shared memory.
template <int N, int PASS, bool MC, int R, int SMX = S_MAX>
__device__ __forceinline__ bool count_item(const CountParams &p, uint32_t tile, uint32_t seg,
                                           uint8_t *smem, uint32_t SB, uint32_t &q) {
    constexpr int NE = EpRegs<N>::NE;
    const uint32_t T = blockDim.x, tid = threadIdx.x;
    uint64_t *bar = stage_bars(smem, SB);
    uint32_t *s_minc = reinterpret_cast<uint32_t *>(smem + 2 * SB + 16);
    uint8_t *ring_raw = smem + 2 * SB + 128;

    const uint32_t ci = tile * T + tid;
    // candidate count: fixed, or produced on the device by an earlier kernel
    const uint32_t m_cur = p.m_dev ? *p.m_dev : p.m;
    if (tile * T >= m_cur) return true;  // the whole block is past the end (uniform)

    // ---------------------------------------------------------------- episode
    EpRegs<N> ep;
    bool ok = ci < m_cur;
    bool distinct = true;  // no type repeats: exactly one node matches any event
    if (ok) {
        const fem_episode rec = p.cands[p.gather ? p.gather[ci] : ci];
        ok = rec.len == N;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            ep.E[k] = rec.types[k];
            ok = ok && ep.E[k] < p.K;
        }
#pragma unroll
        for (int k = 0; k < NE; ++k) {
            ep.lo[k] = 0;
            ep.hi[k] = 0;
            if (k < N - 1) {
                const uint32_t iv = rec.ivl[k];
                ok = ok && iv < p.n_ivl;
                const uint2 b = p.ivl[iv < p.n_ivl ? iv : 0];
                ep.lo[k] = b.x;
                ep.hi[k] = b.y;
            }
        }
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = a + 1; b < N; ++b) distinct = distinct && ep.E[a] != ep.E[b];
        if (MC) ok = ok && distinct;
        if (!ok) atomicOr(p.err, ERR_BADEP);
    }

    // ---------------------------------------------------------------- segment and window
    // A ranged count covers events [ev_begin, ev_end) only: the chunks cr0 .. cr1 - 1,
    // the first from local index lo_local on, the last up to hi_local; its segments
    // are runs of cps chunks from cr0 on, and nothing before ev_begin is read.
    const uint32_t cr0 = p.ranged ? (uint32_t)(p.ev_begin / CHUNK) : 0u;
    const uint32_t cr1 = p.ranged ? (uint32_t)((p.ev_end + CHUNK - 1) / CHUNK) : p.n_chunks;
    const uint32_t c_seg0 = cr0 + seg * p.cps;
    const uint32_t c_end = min(c_seg0 + p.cps, cr1);
    const uint32_t lo_local = p.ranged ? (uint32_t)(p.ev_begin - (uint64_t)cr0 * CHUNK) : 0u;
    const uint32_t hi_local = p.ranged && cr1 > 0
                                  ? (uint32_t)(p.ev_end - (uint64_t)(cr1 - 1) * CHUNK)
                                  : KEY_END;
    const uint64_t L = (uint64_t)c_seg0 * CHUNK;
    // X: start time of the window whose last-node events are the entry classes;
    // X2 = X - W: processing starts there, so that every chain ending inside the
    // window is seen and only window events that can complete an occurrence become
    // classes (the serial machine's last completion before L is one of those).
    uint32_t X = 0, X2 = 0, Xn = 0, c_w = c_seg0;
    bool last_seg = c_end >= cr1;
    if (MC) {
        uint64_t W = 0;
#pragma unroll
        for (int k = 0; k < N - 1; ++k) W += ep.hi[k];
        if (ok && seg > 0) {
            const uint32_t tL = p.cfirst[c_seg0];
            X = (uint64_t)tL >= W ? (uint32_t)(tL - W) : 0u;
            X2 = (uint64_t)tL >= 2 * W ? (uint32_t)(tL - 2 * W) : 0u;
            uint32_t c = c_seg0;
            if (X2 == 0) c = cr0;
            else
                while (c > cr0 && p.cfirst[c] >= X2) --c;
            c_w = c;
        }
        if (!last_seg) {
            const uint32_t tR = p.cfirst[c_end];
            Xn = (uint64_t)tR >= W ? (uint32_t)(tR - W) : 0u;
        }
        if (tid == 0) *s_minc = c_seg0;
        __syncthreads();
        if (ok) atomicMin(s_minc, c_w);
        __syncthreads();
    }
    const uint32_t c_first = MC ? *s_minc : c_seg0;
    const uint32_t q0 = q;

    // ---------------------------------------------------------------- machine state
    uint32_t cnt = 0;
    bool overflow = false, class_overflow = false;
    // relaxed: deadline s + hi + 1 of the latest admitted time per node (0 = unset)
    // and, segmented, the start annotation of that slot
    uint32_t dl[NE], ms[NE];
    // exact: ring cursors plus register copies of each ring's front entry (fx, fy)
    // and back entry (bx, by); the ring itself lives in shared memory
    uint32_t head[NE], tail[NE], fx[NE], fy[NE], bx[NE], by[NE];
#pragma unroll
    for (int k = 0; k < NE; ++k) dl[k] = ms[k] = head[k] = tail[k] = fx[k] = fy[k] = bx[k] = by[k] = 0;
    // MapConcatenate entry classes: class 0 is "none"; class j >= 1 restarts after the
    // last-node event c_key_s[j] of the window.  A class that completes at the same
    // event as class 0 is identical to it from then on: it is merged (its bit in
    // umask cleared, c_cnt[j] holding its count minus class 0's) and no longer updated.
    constexpr int SC = MC ? SMX : 1;  // entry classes per table (SMX slots)
    // used: slots (>= 1) holding a class.  A class that merges into class "none"
    // before the segment starts has the same count and exit as class "none", so its
    // slot is freed: the stitch reads class "none" for any class key not listed.
    uint32_t used = 0, umask = 0;
    // Class keys are written when a class is registered and read for the tables only.
    // From three nodes on they live in shared memory ([slot][thread], after the rings):
    // that frees eight registers where the machine state needs them (level-3 relaxed
    // 0.51 -> 0.47 ms); for two nodes registers are faster.
    constexpr bool KEYS_SMEM = MC && N >= 3;
    uint32_t c_start[SC], c_cnt[SC], c_key[KEYS_SMEM ? 1 : SC];
#pragma unroll
    for (int j = 0; j < SC; ++j) c_start[j] = 0, c_cnt[j] = 0;
#pragma unroll
    for (int j = 0; j < (KEYS_SMEM ? 1 : SC); ++j) c_key[j] = CLS_NONE;
    uint32_t *c_key_s = reinterpret_cast<uint32_t *>(
                            ring_raw + (PASS == FEM_PASS_EXACT && N > 1 ? (size_t)NE * R * T * 8u : 0)) +
                        tid;
    auto set_key = [&](int q0, uint32_t v) {
        if constexpr (KEYS_SMEM) {
            c_key_s[(uint32_t)q0 * T] = v;
        } else {
#pragma unroll
            for (int q = 1; q < SC; ++q)
                if (q == q0) c_key[q] = v;
        }
    };
    auto get_key = [&](int q) -> uint32_t {
        if constexpr (KEYS_SMEM) return q == 0 ? CLS_NONE : c_key_s[(uint32_t)q * T];
        else return c_key[q];
    };
    // Class "none" is a fresh machine at the window start w: it sees chains whose
    // first event is at index >= w, i.e. whose first node's time is >= X.  Until the
    // first node-0 event at or after X its start is unknown and nothing is visible.
    if (MC) c_start[0] = X == 0 ? 0u : 0xFFFFFFFFu;
    bool c0_done = false, capable = false;

    uint2 *ring64 = reinterpret_cast<uint2 *>(ring_raw) + tid;

    // a completion whose chains start no earlier than msv, at event gidx
    auto complete = [&](uint32_t msv, uint32_t gidx) {
        if constexpr (!MC) {
            ++cnt;
        } else {
            const uint32_t inc = (uint64_t)gidx >= L ? 1u : 0u;
            capable = true;
            if (c_start[0] <= msv) c_start[0] = gidx + 1, c_cnt[0] += inc, c0_done = true;
            if (umask) {
#pragma unroll
                for (int j = 1; j < SC; ++j) {
                    if ((umask >> j) & 1u) {
                        if (c_start[j] <= msv) {
                            if (!inc) {
                                // class j says "the serial machine's last completion before
                                // the segment was c_key_s[j]"; a completion before the segment
                                // refutes it, so it is never handed in: drop it
                                used &= ~(1u << j), umask &= ~(1u << j);
                                continue;
                            }
                            c_start[j] = gidx + 1, c_cnt[j] += inc;
                        }
                        if (c_start[j] == c_start[0]) {
                            c_cnt[j] -= c_cnt[0];
                            umask &= ~(1u << j);
                        }
                    }
                }
            }
        }
    };

    auto slot = [&](int q, uint32_t i) -> uint2 & {
        return ring64[((uint32_t)q * R + (i & (R - 1))) * T];
    };
    // drop ring q's front entries that can no longer match (older than hi)
    // Ring entries come in two forms: clusters (first, last) of admitted times whose
    // neighbours are at most hi - lo apart (single-segment machine, and the lean step),
    // or single times with their start annotation (segmented machine before its
    // classes merge).  `cl` selects the form at compile time.
    auto pop_dead_f = [&](auto cl, int q, uint32_t tt) {
        constexpr bool CL = decltype(cl)::value;
        while (head[q] != tail[q] && tt - (CL ? fy[q] : fx[q]) > ep.hi[q]) {
            ++head[q];
            if (head[q] != tail[q]) {
                const uint2 e = slot(q, head[q]);
                fx[q] = e.x, fy[q] = e.y;
            }
        }
    };
    auto push_f = [&](auto cl, int q, uint32_t tt, uint32_t msv) {
        constexpr bool CL = decltype(cl)::value;
        pop_dead_f(cl, q, tt);
        const uint32_t n_in = tail[q] - head[q];
        if (n_in) {
            if (!CL) {
                if (bx[q] == tt) {  // equal times are one entry; annotations only grow
                    by[q] = max(by[q], msv);
                    slot(q, tail[q] - 1u).y = by[q];
                    if (n_in == 1) fy[q] = by[q];
                    return;
                }
            } else if (tt - by[q] <= ep.hi[q] - ep.lo[q]) {  // joins the newest cluster
                by[q] = tt;
                slot(q, tail[q] - 1u).y = tt;
                if (n_in == 1) fy[q] = tt;
                return;
            }
        }
        if (n_in == (uint32_t)R) {
            overflow = true;
            ++head[q];
            const uint2 e = slot(q, head[q]);
            fx[q] = e.x, fy[q] = e.y;
        }
        const uint32_t yv = CL ? tt : msv;
        slot(q, tail[q]) = make_uint2(tt, yv);
        ++tail[q];
        bx[q] = tt, by[q] = yv;
        if (n_in == 0) fx[q] = tt, fy[q] = yv;
    };
    using Clusters = std::integral_constant<bool, true>;
    using Singles = std::integral_constant<bool, !MC>;  // the general step's form
    auto pop_dead = [&](int q, uint32_t tt) { pop_dead_f(Singles{}, q, tt); };
    auto push = [&](int q, uint32_t tt, uint32_t msv) { push_f(Singles{}, q, tt, msv); };

    // One node of the machine for an event at node k (k static after unrolling);
    // returns true when the event completed an occurrence (stop handling it).
    auto step = [&](auto kc, uint32_t tt, uint32_t gidx) -> bool {
        constexpr int k = decltype(kc)::value;
        if constexpr (MC && k == 0) {
            if (c_start[0] == 0xFFFFFFFFu && tt >= X) c_start[0] = gidx;
        }
        if constexpr (N == 1) {
            complete(gidx, gidx);
            return true;
        } else if constexpr (PASS == FEM_PASS_RELAXED) {
            if constexpr (k == 0) {
                dl[0] = tt + ep.hi[0] + 1u;
                if (MC) ms[0] = gidx;
                return false;
            } else {
                if (!(tt < dl[k - 1])) return false;
                if constexpr (k == N - 1) {
                    complete(MC ? ms[k - 1] : 0u, gidx);
                    if (!MC) {
#pragma unroll
                        for (int q = 0; q < NE; ++q) dl[q] = 0;
                    }
                    return true;
                } else {
                    dl[k] = tt + ep.hi[k] + 1u;
                    if (MC) ms[k] = ms[k - 1];
                    return false;
                }
            }
        } else {  // exact
            if constexpr (k == 0) {
                push(0, tt, gidx);
                return false;
            } else {
                constexpr int q = k - 1;
                pop_dead(q, tt);
                if (!(head[q] != tail[q] && tt - fx[q] > ep.lo[q])) return false;
                uint32_t msv = fy[q];
                if (MC) {
                    // annotations grow along the ring: take the newest entry older than lo
                    for (uint32_t i = head[q] + 1u; i != tail[q]; ++i) {
                        const uint2 e = slot(q, i);
                        if (!(tt - e.x > ep.lo[q])) break;
                        msv = e.y;
                    }
                }
                if constexpr (k == N - 1) {
                    complete(msv, gidx);
                    if (!MC) {
#pragma unroll
                        for (int r = 0; r < NE; ++r) head[r] = tail[r];
                    }
                    return true;
                } else {
                    push(k, tt, msv);
                    return false;
                }
            }
        }
    };

    // The same machine step for the common case -- distinct types, event inside the
    // segment proper, every entry class merged into class "none".  With a single class
    // left, an entry is visible iff it was admitted after that class's last
    // completion, so (after purging the entries it cannot see, once) a completion
    // simply empties the state, as in the single-segment machine, and the start
    // annotations are no longer needed.
    auto clear_state = [&]() {
        if constexpr (PASS == FEM_PASS_RELAXED) {
#pragma unroll
            for (int q = 0; q < NE; ++q) dl[q] = 0;
        } else {
#pragma unroll
            for (int q = 0; q < NE; ++q) head[q] = tail[q];
        }
    };
    auto step_lean = [&](auto kc, uint32_t tt, uint32_t gidx) {
        [[maybe_unused]] constexpr int k = decltype(kc)::value;
        auto done_lean = [&]() {
            if constexpr (MC) {
                c_start[0] = gidx + 1, ++c_cnt[0], c0_done = true;
            } else {
                ++cnt;
            }
        };
        if constexpr (N == 1) {
            done_lean();
        } else if constexpr (PASS == FEM_PASS_RELAXED) {
            if constexpr (k == 0) {
                dl[0] = tt + ep.hi[0] + 1u;
            } else if (tt < dl[k - 1]) {
                if constexpr (k == N - 1) {
                    done_lean();
                    clear_state();
                } else {
                    dl[k] = tt + ep.hi[k] + 1u;
                }
            }
        } else {
            if constexpr (k == 0) {
                push_f(Clusters{}, 0, tt, 0u);
            } else {
                constexpr int q = k - 1;
                pop_dead_f(Clusters{}, q, tt);
                if (head[q] != tail[q] && tt - fx[q] > ep.lo[q]) {
                    if constexpr (k == N - 1) {
                        done_lean();
                        clear_state();
                    } else {
                        push_f(Clusters{}, k, tt, 0u);
                    }
                }
            }
        }
    };
    // entering the lean step in the segmented form: drop what class "none" cannot see
    bool purged = !MC;
    auto purge_invisible = [&]() {
        if constexpr (MC) {
            const uint32_t st0 = c_start[0];
            if constexpr (PASS == FEM_PASS_RELAXED) {
#pragma unroll
                for (int q = 0; q < NE; ++q)
                    if (ms[q] < st0) dl[q] = 0;
            } else {
                // annotations grow along each ring: the invisible entries are a prefix;
                // the visible single times are then regrouped into clusters in place
#pragma unroll
                for (int q = 0; q < NE; ++q) {
                    while (head[q] != tail[q] && fy[q] < st0) {
                        ++head[q];
                        if (head[q] != tail[q]) {
                            const uint2 e = slot(q, head[q]);
                            fx[q] = e.x, fy[q] = e.y;
                        }
                    }
                    uint32_t w = head[q];
                    for (uint32_t i = head[q]; i != tail[q]; ++i) {
                        const uint32_t tv2 = slot(q, i).x;
                        if (w != head[q] && tv2 - slot(q, w - 1u).y <= ep.hi[q] - ep.lo[q]) {
                            slot(q, w - 1u).y = tv2;
                        } else {
                            slot(q, w) = make_uint2(tv2, tv2);
                            ++w;
                        }
                    }
                    tail[q] = w;
                    if (head[q] != tail[q]) {
                        const uint2 a = slot(q, head[q]), b = slot(q, tail[q] - 1u);
                        fx[q] = a.x, fy[q] = a.y, bx[q] = b.x, by[q] = b.y;
                    }
                }
            }
        }
    };

    // Two classes whose visible live entries are the same have the same future, even
    // if their starts differ: merge class j into class "none" when no entry that can
    // still match an event at or after time T is visible to one and not the other.
    // Done only while the next segment's window is still more than W ahead (T < Xn),
    // so that both classes hand on the same (normalised) exit.
    auto try_merge = [&](uint32_t T, bool window) {
        if constexpr (MC) {
            if (c_start[0] == 0xFFFFFFFFu || (!last_seg && T >= Xn)) return;
#pragma unroll
            for (int j = 1; j < SC; ++j) {
                if (!((umask >> j) & 1u)) continue;
                const uint32_t lo_s = min(c_start[0], c_start[j]);
                const uint32_t hi_s = max(c_start[0], c_start[j]);
                bool differ = false;
                if constexpr (PASS == FEM_PASS_RELAXED) {
#pragma unroll
                    for (int q = 0; q < NE; ++q)
                        differ |= dl[q] > T && ms[q] >= lo_s && ms[q] < hi_s;
                } else {
#pragma unroll
                    for (int q = 0; q < NE; ++q) {
                        for (uint32_t i = head[q]; i != tail[q] && !differ; ++i) {
                            const uint2 e = slot(q, i);
                            differ = (T < e.x || T - e.x <= ep.hi[q]) && e.y >= lo_s && e.y < hi_s;
                        }
                    }
                }
                if (!differ) {
                    c_cnt[j] -= c_cnt[0];
                    umask &= ~(1u << j);
                    if (window) used &= ~(1u << j);
                }
            }
        }
    };

    // ---------------------------------------------------------------- carried state
    // (single segment only) count and machine state of a count resumed where an
    // earlier call on the same episode stopped
    uint32_t *stw = (!MC && p.state && ok) ? p.state + (uint64_t)ci * p.state_stride : nullptr;
    if (!MC && stw) {
        cnt = stw[0];
        if constexpr (PASS == FEM_PASS_RELAXED) {
#pragma unroll
            for (int k = 0; k < NE; ++k) dl[k] = stw[1 + k];
        } else {
#pragma unroll
            for (int k = 0; k < NE; ++k) {
                const uint32_t *w = stw + 1 + k * (1 + 2 * R);
                const uint32_t nq = min(w[0], (uint32_t)R);
                for (uint32_t i = 0; i < nq; ++i) slot(k, i) = make_uint2(w[1 + 2 * i], w[2 + 2 * i]);
                head[k] = 0;
                tail[k] = nq;
                if (nq) {
                    fx[k] = w[1], fy[k] = w[2];
                    bx[k] = w[2 * nq - 1], by[k] = w[2 * nq];
                }
            }
        }
    }

    // ---------------------------------------------------------------- register rings
    // When every edge of the episode has hi >= 2 lo, consecutive clusters of a list
    // are more than hi - lo >= hi / 2 apart, so a cluster two places behind the
    // newest one ended more than hi before any event that can still come: at most
    // two clusters of each list are live.  The exact pass's lean step then keeps
    // each list as its front (fx, fy) and back (bx, by) cluster plus a count in
    // tail[] (head[] = 0), all in registers: no shared-memory ring traffic.
    constexpr bool EXN = PASS == FEM_PASS_EXACT && N > 1;
    bool ring2 = EXN, in_regs2 = false;
#pragma unroll
    for (int q = 0; q < NE; ++q) ring2 = ring2 && ep.hi[q] - ep.lo[q] >= ep.lo[q];
    auto to_regs2 = [&]() {
#pragma unroll
        for (int q = 0; q < NE; ++q) {
            uint32_t n = tail[q] - head[q];
            if (n > 2) {  // the older clusters have ended (see above)
                const uint2 a = slot(q, tail[q] - 2u);
                fx[q] = a.x, fy[q] = a.y;
                n = 2;
            }
            if (n == 1) bx[q] = fx[q], by[q] = fy[q];
            head[q] = 0, tail[q] = n;
        }
        in_regs2 = true;
    };
    auto from_regs2 = [&]() {
#pragma unroll
        for (int q = 0; q < NE; ++q) {
            if (tail[q] >= 1) slot(q, 0) = make_uint2(fx[q], fy[q]);
            if (tail[q] == 2) slot(q, 1) = make_uint2(bx[q], by[q]);
        }
        in_regs2 = false;
    };

    // ---------------------------------------------------------------- chunk pipeline
    const uint32_t chunk_ev_bytes = CHUNK * 8u;
    const uint32_t chunk_off_bytes = p.offs * 2u;
    auto issue = [&](uint32_t c, uint32_t s) {
        uint8_t *dst = smem + s * SB;
        mbar_expect_tx(&bar[s], chunk_ev_bytes + chunk_off_bytes);
        bulk_g2s(dst, p.bev + (uint64_t)c * CHUNK, chunk_ev_bytes, &bar[s]);
        bulk_g2s(dst + chunk_ev_bytes, p.boff + (uint64_t)c * p.offs, chunk_off_bytes, &bar[s]);
    };
    if (tid == 0) {
        if (c_first < c_end) issue(c_first, q0 & 1u);
        if (c_first + 1 < c_end) issue(c_first + 1, (q0 + 1) & 1u);
    }

    bool bail = false;
    uint32_t c = c_first;
    for (; c < c_end; ++c) {
        const uint32_t j = q0 + (c - c_first), s = j & 1u, par = (j >> 1) & 1u;
        const bool waited = mbar_wait_bounded(&bar[s], par, p.err);
        if (!__syncthreads_and(waited)) {
            bail = true;
            break;
        }
        if (ok && c >= c_w) {
            const uint2 *ev = reinterpret_cast<const uint2 *>(smem + s * SB);
            const uint16_t *off = reinterpret_cast<const uint16_t *>(smem + s * SB + chunk_ev_bytes);
            const uint64_t cbase = (uint64_t)c * CHUNK;
            uint32_t ptr[N], end[N], key[N], tv[N];
#pragma unroll
            for (int k = 0; k < N; ++k) {
                ptr[k] = off[ep.E[k]];
                end[k] = off[ep.E[k] + 1];
                if (MC && c == c_w && X2 > 0)
                    while (ptr[k] < end[k] && ev[ptr[k]].x < X2) ++ptr[k];
                if (c == cr0 && lo_local > 0)
                    while (ptr[k] < end[k] && ev[ptr[k]].y < lo_local) ++ptr[k];
                if (ptr[k] < end[k]) {
                    const uint2 e = ev[ptr[k]];
                    tv[k] = e.x;
                    key[k] = e.y;
                } else {
                    key[k] = KEY_END;
                    tv[k] = 0;
                }
            }
            const uint32_t lim = c + 1 == cr1 ? hi_local : KEY_END;
            bool lean =
                distinct && (!MC || (c >= c_seg0 && umask == 0 && c_start[0] != 0xFFFFFFFFu));
            if (!lean) {
                if (in_regs2) from_regs2();
                uint32_t since = 0;
                for (;;) {
                    uint32_t mk = key[0];
#pragma unroll
                    for (int k = 1; k < N; ++k) mk = min(mk, key[k]);
                    if (mk >= lim) break;
                    const uint32_t gidx = (uint32_t)(cbase + mk);
                    const bool last_hit = key[N - 1] == mk;
                    [[maybe_unused]] const uint32_t t_last = tv[N - 1];  // this event's time if last_hit
                    capable = false;
                    bool done = false;
                    for_nodes_desc<N - 1>([&](auto kc) {
                        constexpr int k = decltype(kc)::value;
                        if (key[k] == mk) {
                            if (!done) done = step(kc, tv[k], gidx);
                            // next entry of this group; reading one past the group's end stays
                            // inside the stage buffer and the value is then discarded
                            ++ptr[k];
                            const uint2 e = ev[ptr[k]];
                            tv[k] = e.x;
                            key[k] = ptr[k] < end[k] ? e.y : KEY_END;
                        }
                    });
                    if (MC && last_hit && capable && (uint64_t)gidx < L &&
                        c_start[0] != gidx + 1) {
                        // entry class r = gidx (the serial machine's last completion was r);
                        // when class "none" completed at r too, it is that class: no slot
                        constexpr uint32_t all_slots = SC >= 32 ? 0xFFFFFFFFu : (1u << SC) - 1u;
                        uint32_t free_slots = ~used & (all_slots & ~1u);
                        if constexpr (PASS == FEM_PASS_EXACT || N >= 4) {
                            if (!free_slots && umask) {
                                // every slot taken: first merge the classes whose futures
                                // have met (a window inside a burst registers many classes
                                // before the chunk's end, where they would otherwise be
                                // merged).  Not in the relaxed kernels of up to three
                                // nodes: the register it takes cost level-3 relaxed 3%.
                                try_merge(t_last, true);
                                free_slots = ~used & (all_slots & ~1u);
                            }
                        }
                        if (free_slots) {
                            const int q0 = __ffs(free_slots) - 1;
                            set_key(q0, gidx);
#pragma unroll
                            for (int q = 1; q < SC; ++q) {
                                if (q == q0) {
                                    c_start[q] = gidx + 1;
                                    c_cnt[q] = 0;
                                }
                            }
                            used |= 1u << q0;
                            umask |= 1u << q0;
                        } else {
                            class_overflow = true;
                        }
                    }
                    // Exact MapConcatenate: classes also merge every 64 events (not only at
                    // chunk ends), and once class "none" is the only one left inside the
                    // segment the rest of the chunk takes the lean step.  (The relaxed
                    // pass keeps chunk-end merges: its general step is cheap, and the extra
                    // registers would cost it occupancy.)
                    if constexpr (MC && PASS == FEM_PASS_EXACT) {
                        if (umask && ++since == 64) {
                            since = 0;
                            uint32_t nk = key[0], nt = tv[0];
#pragma unroll
                            for (int k = 1; k < N; ++k)
                                if (key[k] < nk) nk = key[k], nt = tv[k];
                            if (nk < lim) try_merge(nt, c < c_seg0);
                        }
                        if (distinct && c >= c_seg0 && umask == 0 && c_start[0] != 0xFFFFFFFFu) {
                            lean = true;
                            break;
                        }
                    }
                }
            }
            if (lean) {
                if (!purged) {
                    purge_invisible();
                    purged = true;
                }
                if (EXN && ring2) {
                    if (!in_regs2) to_regs2();
                    for (;;) {
                        uint32_t mk = key[0];
#pragma unroll
                        for (int k = 1; k < N; ++k) mk = min(mk, key[k]);
                        if (mk >= lim) break;
                        lean_nodes<N>(
                            [&](auto kc) { return key[decltype(kc)::value] == mk; },
                            [&](auto kc) {
                            constexpr int k = decltype(kc)::value;
                            {
                                const uint32_t tt = tv[k];
                                // drop list q's clusters that ended more than hi before tt
                                auto pop2 = [&](int q) {
                                    if (tail[q] > 0 && tt - fy[q] > ep.hi[q])
                                        fx[q] = bx[q], fy[q] = by[q], --tail[q];
                                    if (tail[q] > 0 && tt - fy[q] > ep.hi[q]) tail[q] = 0;
                                };
                                // append tt to list q (tail = number of live clusters)
                                auto push2 = [&](int q) {
                                    pop2(q);
                                    const uint32_t n = tail[q];
                                    if (n > 0 && tt - by[q] <= ep.hi[q] - ep.lo[q]) {
                                        by[q] = tt;
                                        if (n == 1) fy[q] = tt;
                                    } else if (n == 0) {
                                        fx[q] = fy[q] = bx[q] = by[q] = tt, tail[q] = 1;
                                    } else if (n == 1) {
                                        bx[q] = by[q] = tt, tail[q] = 2;
                                    } else {  // cannot happen when hi >= 2 lo; reported
                                        overflow = true;
                                        fx[q] = bx[q], fy[q] = by[q], bx[q] = by[q] = tt;
                                    }
                                };
                                if constexpr (k == 0) {
                                    push2(0);
                                } else {
                                    constexpr int q = k - 1;
                                    pop2(q);
                                    if (tail[q] > 0 && tt - fx[q] > ep.lo[q]) {
                                        if constexpr (k == N - 1) {
                                            if constexpr (MC) {
                                                c_start[0] = (uint32_t)(cbase + mk) + 1, ++c_cnt[0],
                                                c0_done = true;
                                            } else {
                                                ++cnt;
                                            }
#pragma unroll
                                            for (int r = 0; r < NE; ++r) tail[r] = 0;
                                        } else {
                                            push2(k);
                                        }
                                    }
                                }
                                ++ptr[k];
                                const uint2 e = ev[ptr[k]];
                                tv[k] = e.x;
                                key[k] = ptr[k] < end[k] ? e.y : KEY_END;
                            }
                        });
                    }
                } else {
                    for (;;) {
                        uint32_t mk = key[0];
#pragma unroll
                        for (int k = 1; k < N; ++k) mk = min(mk, key[k]);
                        if (mk >= lim) break;
                        const uint32_t gidx = (uint32_t)(cbase + mk);
                        for_nodes_desc<N - 1>([&](auto kc) {
                            constexpr int k = decltype(kc)::value;
                            if (key[k] == mk) {
                                step_lean(kc, tv[k], gidx);
                                ++ptr[k];
                                const uint2 e = ev[ptr[k]];
                                tv[k] = e.x;
                                key[k] = ptr[k] < end[k] ? e.y : KEY_END;
                            }
                        });
                    }
                }
            }
            if (MC && umask) try_merge(p.cfirst[c + 1], c < c_seg0);
        }
        __syncthreads();
        if (tid == 0 && c + 2 < c_end) {
            fence_proxy_async_smem();
            issue(c + 2, s);
        }
    }
    if (bail) {
        // drain the copies still in flight before the block's shared memory goes away
        if (tid == 0) {
            for (uint32_t cc = c; cc < min(c + 2, c_end); ++cc) {
                const uint32_t j = q0 + (cc - c_first);
                mbar_wait_bounded(&bar[j & 1u], (j >> 1) & 1u, p.err);
            }
        }
        return false;
    }
    q = q0 + (c_end > c_first ? c_end - c_first : 0u);

    // ---------------------------------------------------------------- results
    if (ci >= m_cur) return true;
    if (overflow || class_overflow) {
        atomicOr(p.err, (overflow ? ERR_RING : 0u) | (class_overflow ? ERR_CLASS : 0u));
        p.redo[ci] = 1;
    }
    if (in_regs2) from_regs2();
    if (!MC && stw) {
        stw[0] = cnt;
        if constexpr (PASS == FEM_PASS_RELAXED) {
#pragma unroll
            for (int k = 0; k < NE; ++k) stw[1 + k] = dl[k];
        } else {
#pragma unroll
            for (int k = 0; k < NE; ++k) {
                uint32_t *w = stw + 1 + k * (1 + 2 * R);
                const uint32_t nq = tail[k] - head[k];
                w[0] = nq;
                for (uint32_t i = 0; i < nq; ++i) {
                    const uint2 e = slot(k, head[k] + i);
                    w[1 + 2 * i] = e.x;
                    w[2 + 2 * i] = e.y;
                }
            }
        }
    }
    if (!MC) {
        p.out[ci] = ok ? cnt : 0u;
    } else {
        // slots 0 .. n-1 are written (n = 1 + the highest used slot, in slot 0's w);
        // the stitch reads no further
        uint4 *tab = p.tables + ((uint64_t)seg * p.m + ci) * SMX;
        const uint32_t n_slots = used ? 32u - __clz(used) : 1u;
#pragma unroll
        for (int q = 0; q < SMX; ++q) {
            if ((uint32_t)q >= n_slots) break;
            uint4 e = make_uint4(CLS_EMPTY, 0, CLS_NONE, q == 0 ? n_slots : 0u);
            if (ok && (q == 0 || ((used >> q) & 1u))) {
                const bool merged = q > 0 && !((umask >> q) & 1u);
                const uint32_t cntq = merged ? c_cnt[0] + c_cnt[q] : c_cnt[q];
                const uint32_t st = merged ? c_start[0] : c_start[q];
                // the last completion (or the class's own event) is st - 1; it is
                // handed on only if it lies in the next segment's window
                uint32_t ex = (q == 0 && !c0_done) ? CLS_NONE : st - 1u;
                if (ex != CLS_NONE && !last_seg && p.t[ex] < Xn) ex = CLS_NONE;
                e = make_uint4(get_key(q), cntq, ex, q == 0 ? n_slots : 0u);
            }
            tab[q] = e;
        }
    }
    return true;
}

__device__ __forceinline__ void init_stage_bars(uint8_t *smem, uint32_t SB) {
    if (threadIdx.x == 0) {
        uint64_t *bar = stage_bars(smem, SB);
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
}

// One block per (episode tile, segment) of one candidate set.  Three register
// budgets, each the fastest measured for its kernels: the compiler's default for the
// relaxed pass up to three nodes (64 registers keep four 256-thread blocks per SM);
// three blocks per SM for the exact pass with two nodes; and one block's worth for
// longer episodes, whose class tables and lists otherwise land in local memory
// (level-5 relaxed on the 11.8M-event stream: 170 -> 71 ms).
template <int N, int PASS, bool MC, int R, int SMX>
__device__ __forceinline__ void count_block(const CountParams &p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t SB = stage_bytes(p.offs);
    init_stage_bars(smem, SB);
    uint32_t q = 0;
    count_item<N, PASS, MC, R, SMX>(p, blockIdx.x, blockIdx.y, smem, SB, q);
}

// SMX: entry-class slots per transfer table (more for the recount of episodes whose
// first count ran out of slots)
template <int N, int PASS, bool MC, int R, int SMX>
__global__ void __launch_bounds__(256) k_count(const CountParams p) {
    count_block<N, PASS, MC, R, SMX>(p);
}

template <int N, int PASS, bool MC, int R, int SMX>
__global__ void __launch_bounds__(256, 3) k_count_exact(const CountParams p) {
    count_block<N, PASS, MC, R, SMX>(p);
}

template <int N, int PASS, bool MC, int R, int SMX>
__global__ void __launch_bounds__(256, 1) k_count_wide(const CountParams p) {
    count_block<N, PASS, MC, R, SMX>(p);
}

// Persistent form for a batch of candidate sets over several streams: each block
// takes (job, tile, segment) items from a device queue until the list is
// exhausted.  Items come longest first; `jobs` and the item list are device
// resident, so a captured graph can replay the launch with new sizes.
template <int N, int PASS, bool MC, int R>
__device__ __forceinline__ void count_batch_loop(const CountParams *__restrict__ jobs,
                                                 const uint4 *__restrict__ items,
                                                 const uint32_t *n_items, uint32_t *queue,
                                                 uint32_t SB) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ CountParams s_job;
    __shared__ uint32_t s_item;
    init_stage_bars(smem, SB);
    uint32_t q = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= *n_items) break;
        const uint4 d = items[it];
        if (threadIdx.x == 0) s_job = jobs[d.x];
        __syncthreads();
        if (!count_item<N, PASS, MC, R>(s_job, d.y, d.z, smem, SB, q)) break;
        __syncthreads();
    }
}

template <int N, int PASS, bool MC, int R>
__global__ void __launch_bounds__(256) k_count_batch(const CountParams *__restrict__ jobs,
                                                     const uint4 *__restrict__ items,
                                                     const uint32_t *n_items, uint32_t *queue,
                                                     uint32_t SB) {
    count_batch_loop<N, PASS, MC, R>(jobs, items, n_items, queue, SB);
}

template <int N, int PASS, bool MC, int R>
__global__ void __launch_bounds__(256, 3)
    k_count_batch_exact(const CountParams *__restrict__ jobs, const uint4 *__restrict__ items,
                        const uint32_t *n_items, uint32_t *queue, uint32_t SB) {
    count_batch_loop<N, PASS, MC, R>(jobs, items, n_items, queue, SB);
}

template <int N, int PASS, bool MC, int R>
__global__ void __launch_bounds__(256, 1)
    k_count_batch_wide(const CountParams *__restrict__ jobs, const uint4 *__restrict__ items,
                       const uint32_t *n_items, uint32_t *queue, uint32_t SB) {
    count_batch_loop<N, PASS, MC, R>(jobs, items, n_items, queue, SB);
}

// The kernel (register budget) of a (N, pass, MC, R) instantiation.
template <int N, int PASS>
constexpr int count_budget() {  // 0: compiler default, 3: three blocks per SM, 1: one
    return PASS == FEM_PASS_EXACT ? (N <= 2 ? 3 : 1) : (N <= 3 ? 0 : 1);
}
template <int N, int PASS, bool MC, int R, int SMX = S_MAX>
constexpr auto count_kernel() {
    if constexpr (SMX > S_MAX) return k_count_wide<N, PASS, MC, R, SMX>;  // recount tables
    else if constexpr (count_budget<N, PASS>() == 3) return k_count_exact<N, PASS, MC, R, SMX>;
    else if constexpr (count_budget<N, PASS>() == 1) return k_count_wide<N, PASS, MC, R, SMX>;
    else return k_count<N, PASS, MC, R, SMX>;
}
template <int N, int PASS, bool MC, int R>
constexpr auto count_batch_kernel() {
    if constexpr (count_budget<N, PASS>() == 3) return k_count_batch_exact<N, PASS, MC, R>;
    else if constexpr (count_budget<N, PASS>() == 1) return k_count_batch_wide<N, PASS, MC, R>;
    else return k_count_batch<N, PASS, MC, R>;
}

}  // namespace fem
