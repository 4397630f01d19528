// fem_windows.cu -- window-based frequency (the alternative measure Section 2 names,
// after Mannila et al.), with the episode's interval constraints: the number of
// integer window starts s such that some occurrence lies inside [s, s + w).
//
// One thread per episode walks the bucketed stream (global memory, L2-resident for
// the workloads here), merging its N type groups by local index.  For each event j
// of node k it needs L_k(j), the latest first-node time over the chains ending at j:
// the maximum of L_{k-1} over the node-(k-1) events i < j with lo < t[j] - t[i] <= hi.
// Per edge that is a sliding-window maximum: entries (t, L) of node k-1 wait in a
// FIFO until they are older than lo, then enter a deque kept decreasing in L (an
// entry behind a larger, newer one can never be the maximum again), whose front is
// dropped once older than hi.  A last-node event with L defined covers the starts
// (t[j] - w, L]; these ranges come in order of their left ends and are merged on
// the fly.
#include "fem_internal.cuh"

namespace fem {

namespace {

constexpr int WQ = 32;  // entries per FIFO and per deque

template <int N>
__global__ void __launch_bounds__(128) k_count_windows(const WindowParams p) {
    constexpr int NE = N > 1 ? N - 1 : 1;
    const uint32_t ci = blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= p.m) return;
    const fem_episode rec = p.cands[ci];
    if (rec.len != N) return;
    uint32_t E[N], lo[NE], hi[NE];
#pragma unroll
    for (int q = 0; q < N; ++q) E[q] = rec.types[q];
#pragma unroll
    for (int q = 0; q < NE; ++q) {
        lo[q] = hi[q] = 0;
        if (q < N - 1) {
            const uint2 b = p.ivl[rec.ivl[q]];
            lo[q] = b.x, hi[q] = b.y;
        }
    }
    // per edge q: FIFO (entries of node q not yet older than lo) and deque
    uint32_t ft[NE][WQ], fl[NE][WQ], fh[NE], fn[NE];
    uint32_t dt[NE][WQ], dl[NE][WQ], dh[NE], dn[NE];
#pragma unroll
    for (int q = 0; q < NE; ++q) fh[q] = fn[q] = dh[q] = dn[q] = 0;
    bool overflow = false;
    auto fifo_push = [&](int q, uint32_t tt, uint32_t L) {
        if (fn[q] == WQ) {
            overflow = true;
            return;
        }
        const uint32_t at = (fh[q] + fn[q]) % WQ;
        ft[q][at] = tt, fl[q][at] = L;
        ++fn[q];
    };
    // the latest first-node time over the chains reaching an event at time tt
    // through edge q (false if there is none)
    auto window_max = [&](int q, uint32_t tt, uint32_t *out) -> bool {
        while (fn[q] && tt - ft[q][fh[q]] > lo[q]) {
            const uint32_t t1 = ft[q][fh[q]], L1 = fl[q][fh[q]];
            fh[q] = (fh[q] + 1) % WQ, --fn[q];
            while (dn[q] && dl[q][(dh[q] + dn[q] - 1) % WQ] <= L1) --dn[q];
            if (dn[q] == WQ) {
                overflow = true;
                continue;
            }
            const uint32_t at = (dh[q] + dn[q]) % WQ;
            dt[q][at] = t1, dl[q][at] = L1;
            ++dn[q];
        }
        while (dn[q] && tt - dt[q][dh[q]] > hi[q]) dh[q] = (dh[q] + 1) % WQ, --dn[q];
        if (!dn[q]) return false;
        *out = dl[q][dh[q]];
        return true;
    };

    const int64_t w = p.w;
    uint64_t total = 0;
    int64_t cur_a = 0, cur_b = -1;
    bool have = false;
    const uint32_t n_chunks = (uint32_t)((p.n + CHUNK - 1) / CHUNK);
    for (uint32_t c = 0; c < n_chunks; ++c) {
        const uint16_t *off = p.boff + (uint64_t)c * p.offs;
        const uint2 *ev = p.bev + (uint64_t)c * CHUNK;
        uint32_t ptr[N], end[N];
#pragma unroll
        for (int q = 0; q < N; ++q) ptr[q] = off[E[q]], end[q] = off[E[q] + 1];
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
            uint32_t L = tt;
            bool defined = true;
            if (kq > 0) defined = window_max(kq - 1, tt, &L);
            if (!defined) continue;
            if (kq < N - 1) {
                fifo_push(kq, tt, L);
                continue;
            }
            const int64_t a = (int64_t)tt - w + 1, b = (int64_t)L;
            if (a > b) continue;  // every chain ending here is longer than the window
            if (have && a <= cur_b + 1) {
                if (b > cur_b) cur_b = b;
            } else {
                if (have) total += (uint64_t)(cur_b - cur_a + 1);
                cur_a = a, cur_b = b, have = true;
            }
        }
    }
    if (have) total += (uint64_t)(cur_b - cur_a + 1);
    if (overflow) atomicOr(p.err, ERR_RING);
    p.out[ci] = total;
}

template <int N>
cudaError_t windows_n(const WindowParams &p, cudaStream_t st) {
    k_count_windows<N><<<(p.m + 127) / 128, 128, 0, st>>>(p);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_count_windows(const WindowParams &p, uint32_t len_mask, cudaStream_t st) {
    if (p.m == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (len_mask & (1u << 1)) e = windows_n<1>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 2))) e = windows_n<2>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 3))) e = windows_n<3>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 4))) e = windows_n<4>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 5))) e = windows_n<5>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 6))) e = windows_n<6>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 7))) e = windows_n<7>(p, st);
    if (e == cudaSuccess && (len_mask & (1u << 8))) e = windows_n<8>(p, st);
    return e;
}

}  // namespace fem
