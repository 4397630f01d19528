// fem_literal.cu -- MapConcatenate as Section 5.2.2 prints it, kept beside the exact
// reformulation of fem_count.cuh as a measured comparison.
//
// Segments are time ranges (tau[p], tau[p+1]].  For each (episode, segment p,
// machine k < N) one thread runs Algorithm 1 (windowed lists, stored as clusters as
// in the exact counter) on the events with t > tau[p] - (hi[0] + ... + hi[k-1]):
// it counts the completions inside the segment, records a = the end time of its
// first completion in (tau[p], tau[p] + W) and, past the segment's end, advances
// only the partial occurrences it holds (node 0 admits nothing) over the events with
// t < tau[p+1] + W, recording b = the end time of the first completion there.  A
// second kernel joins, per episode and from machine 0 of segment 0, each segment's
// tuple to the next segment's tuple whose a equals its b (smallest k when several do,
// k = 0 when none does), summing the counts.
//
// Events are read straight from the bucketed stream in global memory (L2-resident
// for the workloads here); lists live in per-thread local memory.  This variant is
// for comparison: its counts differ from the exact ones where the printed scheme
// loses occurrences, and it does N times the machine work of one segment.
#include "fem_internal.cuh"

namespace fem {

namespace {

constexpr int LR = 16;  // clusters per list

__device__ __forceinline__ uint64_t first_after(const uint32_t *t, uint64_t n, int64_t x) {
    uint64_t a = 0, b = n;
    while (a < b) {
        const uint64_t mid = a + (b - a) / 2;
        if ((int64_t)t[mid] > x) b = mid;
        else a = mid + 1;
    }
    return a;
}

// tuples[(ci * P + seg) * FEM_MAX_LEN + k] = (a, count, b, bit 0: a set, bit 1: b set)
template <int N>
__global__ void __launch_bounds__(128) k_literal_map(const LiteralParams p) {
    constexpr int NE = N > 1 ? N - 1 : 1;
    const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t k = (uint32_t)(idx % N);
    const uint64_t r = idx / N;
    const uint32_t seg = (uint32_t)(r % p.P);
    const uint64_t ci = r / p.P;
    if (ci >= p.m) return;
    const fem_episode rec = p.cands[ci];
    if (rec.len != N) return;
    uint32_t E[N], lo[NE], hi[NE];
    int64_t W = 0, back = 0;
#pragma unroll
    for (int q = 0; q < N; ++q) E[q] = rec.types[q];
#pragma unroll
    for (int q = 0; q < NE; ++q) {
        lo[q] = hi[q] = 0;
        if (q < N - 1) {
            const uint2 b = p.ivl[rec.ivl[q]];
            lo[q] = b.x, hi[q] = b.y;
            W += b.y;
            if ((uint32_t)q < k) back += b.y;
        }
    }
    const int64_t tauA = p.tau[seg], tauB = p.tau[seg + 1];
    const int64_t endB = tauB + W;

    // lists of clusters (first, last), ring per edge
    uint32_t cf[NE][LR], cl[NE][LR], head[NE], cnt_q[NE];
#pragma unroll
    for (int q = 0; q < NE; ++q) head[q] = cnt_q[q] = 0;
    bool overflow = false;
    auto pop_dead = [&](int q, uint32_t tt) {
        while (cnt_q[q] && tt - cl[q][head[q]] > hi[q]) head[q] = (head[q] + 1) % LR, --cnt_q[q];
    };
    auto push = [&](int q, uint32_t tt) {
        pop_dead(q, tt);
        if (cnt_q[q]) {
            const uint32_t bk = (head[q] + cnt_q[q] - 1) % LR;
            if (tt - cl[q][bk] <= hi[q] - lo[q]) {
                cl[q][bk] = tt;
                return;
            }
        }
        if (cnt_q[q] == LR) {
            overflow = true;
            return;
        }
        const uint32_t at = (head[q] + cnt_q[q]) % LR;
        cf[q][at] = cl[q][at] = tt;
        ++cnt_q[q];
    };

    uint32_t count = 0, a = 0, b = 0, flags = 0;
    bool stop = false;
    const uint64_t i0 = first_after(p.t, p.n, tauA - back);
    const uint32_t n_chunks = (uint32_t)((p.n + CHUNK - 1) / CHUNK);
    for (uint32_t c = (uint32_t)(i0 / CHUNK); c < n_chunks && !stop; ++c) {
        const uint16_t *off = p.boff + (uint64_t)c * p.offs;
        const uint2 *ev = p.bev + (uint64_t)c * CHUNK;
        const uint32_t lo_local = c == (uint32_t)(i0 / CHUNK) ? (uint32_t)(i0 - (uint64_t)c * CHUNK) : 0u;
        uint32_t ptr[N], end[N];
#pragma unroll
        for (int q = 0; q < N; ++q) {
            ptr[q] = off[E[q]];
            end[q] = off[E[q] + 1];
            while (ptr[q] < end[q] && ev[ptr[q]].y < lo_local) ++ptr[q];
        }
        for (;;) {
            uint32_t mk = KEY_END;
            int kq = -1;
#pragma unroll
            for (int q = 0; q < N; ++q) {
                if (ptr[q] < end[q]) {
                    const uint32_t y = ev[ptr[q]].y;
                    if (y < mk) mk = y, kq = q;
                }
            }
            if (kq < 0) break;
            uint32_t tt = 0;
#pragma unroll
            for (int q = 0; q < N; ++q)
                if (q == kq) tt = ev[ptr[q]].x, ++ptr[q];
            const bool phase2 = (int64_t)tt > tauB;
            if (phase2 && (int64_t)tt >= endB) {
                stop = true;
                break;
            }
            bool done = false;
            if (kq == 0) {
                if (N == 1) done = !phase2;
                else if (!phase2) push(0, tt);
            } else {
                const int q = kq - 1;
                pop_dead(q, tt);
                if (cnt_q[q] && tt - cf[q][head[q]] > lo[q]) {
                    if (kq == N - 1) {
                        done = true;
#pragma unroll
                        for (int z = 0; z < NE; ++z) cnt_q[z] = 0;
                    } else {
                        push(kq, tt);
                    }
                }
            }
            if (!done) continue;
            if (phase2) {
                b = tt, flags |= 2u;
                stop = true;
                break;
            }
            if ((int64_t)tt > tauA) {
                ++count;
                if (!(flags & 1u) && (int64_t)tt < tauA + W) a = tt, flags |= 1u;
            }
        }
    }
    if (overflow) atomicOr(p.err, ERR_RING);
    p.tuples[(ci * p.P + seg) * FEM_MAX_LEN + k] = make_uint4(a, count, b, flags);
}

// Concatenate, left to right per episode (equal to the paper's pairwise tree when
// each boundary has one choice).
__global__ void k_literal_join(const LiteralParams p, uint32_t *out, uint32_t *diag) {
    const uint32_t ci = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t none = 0, several = 0;
    if (ci < p.m) {
        const uint32_t N = p.cands[ci].len;
        const uint4 *tp = p.tuples + (uint64_t)ci * p.P * FEM_MAX_LEN;
        uint4 cur = tp[0];
        uint32_t total = cur.y;
        for (uint32_t s = 1; s < p.P; ++s) {
            const uint4 *row = tp + (uint64_t)s * FEM_MAX_LEN;
            const bool b_set = (cur.w & 2u) != 0;
            int pick = -1, hits = 0;
            for (uint32_t k = 0; k < N; ++k) {
                const bool a_set = (row[k].w & 1u) != 0;
                if (a_set == b_set && (!a_set || row[k].x == cur.z)) {
                    ++hits;
                    if (pick < 0) pick = (int)k;
                }
            }
            if (hits == 0) ++none, pick = 0;
            if (hits > 1) ++several;
            cur = row[pick];
            total += cur.y;
        }
        out[ci] = total;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        none += __shfl_down_sync(0xFFFFFFFFu, none, o);
        several += __shfl_down_sync(0xFFFFFFFFu, several, o);
    }
    if ((threadIdx.x & 31u) == 0) {
        if (none) atomicAdd(&diag[0], none);
        if (several) atomicAdd(&diag[1], several);
    }
}

template <int N>
cudaError_t map_n(const LiteralParams &p, cudaStream_t st) {
    const uint64_t threads = (uint64_t)p.m * p.P * N;
    if (!threads) return cudaSuccess;
    const uint64_t blocks = (threads + 127) / 128;
    if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
    k_literal_map<N><<<(uint32_t)blocks, 128, 0, st>>>(p);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_literal(const LiteralParams &p, uint32_t len_mask, uint32_t *out, uint32_t *diag,
                           cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (len_mask & (1u << 1)) e = map_n<1>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 2))) e = map_n<2>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 3))) e = map_n<3>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 4))) e = map_n<4>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 5))) e = map_n<5>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 6))) e = map_n<6>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 7))) e = map_n<7>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 8))) e = map_n<8>(p, st);
    if (e != cudaSuccess) return e;
    k_literal_join<<<(p.m + 255) / 256, 256, 0, st>>>(p, out, diag);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fem
