"""Seeded synthetic spike-train workloads (inputs only; no counting arithmetic).

Every generator draws from ``numpy.random.Generator(PCG64(seed))`` and returns
plain arrays, so the CUDA path and the CPU oracle are fed identical inputs.
The streams stand in for the paper's Sym26 simulation and its cortical-culture
recordings (Section 6.1), which are not available: each neuron (event type)
fires as a homogeneous Poisson process, and a few causal chains are embedded
as cascades (a trigger fires the chain's first neuron, each next neuron fires
after a delay drawn inside one of the interval set's intervals).

Times are integer microseconds (uint32).  Events are ordered by time, ties by
type, then by emission order, which is the order every consumer must keep.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LMAX = 8

# Interval set of the 64-type workloads: (0,2], (2,5], (5,10], (10,20] ms, in microseconds.
I_MS4 = np.array([[0, 2000], [2000, 5000], [5000, 10000], [10000, 20000]], np.uint32)


@dataclass
class Stream:
    types: np.ndarray          # uint8[n]
    t: np.ndarray              # uint32[n], non-decreasing
    n_types: int
    chains: list = field(default_factory=list)   # [(types tuple, interval-index tuple, rate Hz)]

    @property
    def n(self) -> int:
        return int(self.t.shape[0])


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def poisson_stream(seed, n_types, rates_hz, duration_s, chains=(), delay_fn=None):
    """Background Poisson firing plus embedded cascades.

    rates_hz: scalar or float[n_types].  chains: iterable of
    (types tuple, trigger rate Hz, per-edge (lo, hi) microsecond ranges);
    each trigger at t0 emits types[0] at t0 and types[k+1] at
    t_k + d_k, d_k drawn by ``delay_fn(rng, lo, hi)`` (default: the interval
    midpoint plus integer jitter in [-500, 500] µs, clipped inside (lo, hi]).
    Events past the duration are dropped.
    """
    rng = _rng(seed)
    T_us = int(round(duration_s * 1e6))
    rates = np.broadcast_to(np.asarray(rates_hz, dtype=np.float64), (n_types,))
    ts, ty = [], []
    for a in range(n_types):
        k = rng.poisson(rates[a] * duration_s)
        ts.append(np.floor(rng.random(k) * T_us).astype(np.int64))
        ty.append(np.full(k, a, np.int64))
    if delay_fn is None:
        def delay_fn(r, lo, hi, size):
            mid = (int(lo) + int(hi)) // 2
            d = mid + r.integers(-500, 501, size=size)
            return np.clip(d, int(lo) + 1, int(hi))
    for ctypes_, rate, edges in chains:
        k = rng.poisson(rate * duration_s)
        t0 = np.floor(rng.random(k) * T_us).astype(np.int64)
        cur = t0
        ts.append(cur)
        ty.append(np.full(k, ctypes_[0], np.int64))
        for j, (lo, hi) in enumerate(edges):
            cur = cur + delay_fn(rng, lo, hi, k)
            ts.append(cur.copy())
            ty.append(np.full(k, ctypes_[j + 1], np.int64))
    t_all = np.concatenate(ts) if ts else np.zeros(0, np.int64)
    ty_all = np.concatenate(ty) if ty else np.zeros(0, np.int64)
    emit = np.arange(t_all.shape[0])
    keep = t_all < T_us
    t_all, ty_all, emit = t_all[keep], ty_all[keep], emit[keep]
    order = np.lexsort((emit, ty_all, t_all))
    return t_all[order].astype(np.uint32), ty_all[order].astype(np.uint8)


def chance_theta(rate_hz, duration_s, window_s, factor=5.0, power=1):
    """ceil(factor * rate*T * (1 - exp(-rate*window))**power): a support threshold
    set at `factor` times a Poisson chance count (the workload's stated rule)."""
    return int(math.ceil(factor * rate_hz * duration_s * (1 - math.exp(-rate_hz * window_s)) ** power))


# --------------------------------------------------------------------------- named workloads
def tiny_mining(seed=0xFE01):
    """16 types at 20 Hz for 10 s, cascade 0->1->2->3 at 2 Hz with delays uniform in
    [4500, 5500] µs; interval set {(4,6] ms}; threshold 15; mined to length 4."""
    def uni(r, lo, hi, size):
        return r.integers(4500, 5501, size=size)
    t, ty = poisson_stream(seed, 16, 20.0, 10.0,
                           chains=[((0, 1, 2, 3), 2.0, [(4000, 6000)] * 3)], delay_fn=uni)
    I = np.array([[4000, 6000]], np.uint32)
    return dict(name="tiny_mining_16types_10s", stream=Stream(ty, t, 16, [((0, 1, 2, 3), (0, 0, 0), 2.0)]),
                intervals=I, theta=15, max_len=4)


def _chains(rng, n_chains, n_types, lens, n_int, rate_lo, rate_hi):
    out = []
    for _ in range(n_chains):
        L = int(rng.choice(lens))
        tys = tuple(int(x) for x in rng.choice(n_types, size=L, replace=False))
        ivs = tuple(int(x) for x in rng.integers(0, n_int, size=L - 1))
        rate = float(rng.uniform(rate_lo, rate_hi))
        out.append((tys, ivs, rate))
    return out


def single_recording(seed=0xFE02, deep=False):
    """64 types at 20 Hz for 300 s with 8 chains (lengths 4-6, 1-3 Hz, delays inside
    intervals of I_MS4 with +-0.5 ms jitter); level-2 candidates 64*63*4 = 16,128;
    mined to length 6.  Threshold: 5x the chance count of the narrowest interval
    (1177), or 300 for the deep variant."""
    rng = _rng(seed + 0x100)
    ch = _chains(rng, 8, 64, [4, 5, 6], len(I_MS4), 1.0, 3.0)
    spec = [(tys, rate, [tuple(I_MS4[i]) for i in ivs]) for tys, ivs, rate in ch]
    t, ty = poisson_stream(seed, 64, 20.0, 300.0, chains=spec)
    theta = 300 if deep else chance_theta(20.0, 300.0, 0.002)
    return dict(name="single_recording_64types_300s" + ("_deep" if deep else ""),
                stream=Stream(ty, t, 64, ch), intervals=I_MS4.copy(), theta=theta, max_len=6)


# Interval set of the bursty workload: I_MS4's first three plus (15,20] ms, whose
# hi < 2 lo lets more than two clusters of a list be live (the shared-memory rings).
I_BURST = np.array([[0, 2000], [2000, 5000], [5000, 10000], [15000, 20000]], np.uint32)


def bursty_recording(seed=0xFE06, n_types=64, duration_s=300.0, base_hz=5.0,
                     burst_hz=0.5, burst_ms=(50.0, 200.0), burst_rate_hz=200.0):
    """A network-bursting culture: every type fires at `base_hz`, and network bursts
    (Poisson, `burst_hz`; duration uniform in `burst_ms`) make every type fire at
    `burst_rate_hz` for the burst's length; 8 chains of 4-6 nodes at 1-3 Hz with
    delays inside I_BURST.  Candidates: all 16,128 ordered pairs x I_BURST plus 20,000
    random episodes of 3-4 nodes; threshold 5x the chance count of the narrowest
    interval at the mean rate (903), which most pairs pass inside bursts, so the exact
    pass (Algorithm 4's second pass) runs on most of them."""
    rng = _rng(seed + 0x100)
    ch = _chains(rng, 8, n_types, [4, 5, 6], len(I_BURST), 1.0, 3.0)
    spec = [(tys, rate, [tuple(I_BURST[i]) for i in ivs]) for tys, ivs, rate in ch]
    t, ty = poisson_stream(seed, n_types, base_hz, duration_s, chains=spec)
    # bursts: per burst, every type a Poisson count over its span
    T_us = int(round(duration_s * 1e6))
    nb = rng.poisson(burst_hz * duration_s)
    b0 = np.floor(rng.random(nb) * T_us).astype(np.int64)
    blen = (rng.uniform(burst_ms[0], burst_ms[1], nb) * 1000).astype(np.int64)
    bt, bty = [], []
    for start, ln in zip(b0, blen):
        k = rng.poisson(burst_rate_hz * ln * 1e-6, size=n_types)
        tot = int(k.sum())
        bt.append(start + np.floor(rng.random(tot) * ln).astype(np.int64))
        bty.append(np.repeat(np.arange(n_types), k))
    if nb:
        t2 = np.concatenate([t.astype(np.int64)] + bt)
        ty2 = np.concatenate([ty.astype(np.int64)] + bty)
        emit = np.arange(t2.shape[0])
        keep = t2 < T_us
        t2, ty2, emit = t2[keep], ty2[keep], emit[keep]
        order = np.lexsort((emit, ty2, t2))
        t, ty = t2[order].astype(np.uint32), ty2[order].astype(np.uint8)
    mean_hz = base_hz + burst_hz * np.mean(burst_ms) * 1e-3 * burst_rate_hz
    theta = chance_theta(mean_hz, duration_s, 0.002)
    L2, E2, iv2 = level2_candidates(range(n_types), len(I_BURST))
    L3, E3, iv3 = random_candidates(seed + 0x200, 20_000, n_types, [3, 4], len(I_BURST))
    cands = (np.concatenate([L2, L3]), np.concatenate([E2, E3]), np.concatenate([iv2, iv3]))
    return dict(name=f"bursty_recording_{n_types}types_{int(duration_s)}s",
                stream=Stream(ty, t, n_types, ch), intervals=I_BURST.copy(), theta=theta,
                candidates=cands, bursts=(b0, blen))


def sparse_bursts(seed=3, n_types=16, base_hz=5.0, duration_s=300.0, n_bursts=6,
                  burst_ms=100.0, burst_rate_hz=200.0):
    """A quiet Poisson stream (every type at `base_hz`) with `n_bursts` bursts of
    `burst_ms` each, at uniform times, in which every type fires at `burst_rate_hz`.
    Returns (types uint8[n], t uint32[n]), sorted by time (ties by type)."""
    t, ty = poisson_stream(seed, n_types, base_hz, duration_s)
    rng = np.random.default_rng(seed)
    T_us = int(round(duration_s * 1e6))
    ln = int(round(burst_ms * 1000))
    bt, bty = [t.astype(np.int64)], [ty.astype(np.int64)]
    for _ in range(n_bursts):
        start = int(rng.integers(T_us // 300, T_us - T_us // 300))
        k = rng.poisson(burst_rate_hz * burst_ms * 1e-3, size=n_types)
        bt.append(start + np.floor(rng.random(int(k.sum())) * ln).astype(np.int64))
        bty.append(np.repeat(np.arange(n_types), k))
    t2, ty2 = np.concatenate(bt), np.concatenate(bty)
    order = np.lexsort((ty2, t2))
    return ty2[order].astype(np.uint8), t2[order].astype(np.uint32)


def large_stream(seed=0xFE04, n_candidates=100_000, duration_s=3600.0):
    """64 types at 50 Hz for 1 h plus 8 chains; 100k random candidates of lengths 3-5
    with distinct types and random intervals from I_MS4; threshold 5x the chance
    count of the narrowest length-3 episode."""
    rng = _rng(seed + 0x100)
    ch = _chains(rng, 8, 64, [4, 5, 6], len(I_MS4), 1.0, 3.0)
    spec = [(tys, rate, [tuple(I_MS4[i]) for i in ivs]) for tys, ivs, rate in ch]
    t, ty = poisson_stream(seed, 64, 50.0, duration_s, chains=spec)
    cands = random_candidates(seed + 0x200, n_candidates, 64, [3, 4, 5], len(I_MS4))
    theta = chance_theta(50.0, duration_s, 0.002, power=2)
    return dict(name=f"large_stream_64types_{int(duration_s)}s", stream=Stream(ty, t, 64, ch),
                intervals=I_MS4.copy(), theta=theta, candidates=cands)


def random_candidates(seed, m, n_types, lens, n_int, distinct=True):
    """m random episodes: (len uint8[m], types uint8[m,8], ivl uint8[m,7]); lengths drawn
    from `lens`, types distinct within an episode (unless distinct=False), interval
    indices uniform."""
    rng = _rng(seed)
    L = rng.choice(np.asarray(lens), size=m).astype(np.uint8)
    E = np.zeros((m, LMAX), np.uint8)
    iv = np.zeros((m, LMAX - 1), np.uint8)
    for a in range(0, m, 65536):
        b = min(m, a + 65536)
        if distinct:
            pick = np.argsort(rng.random((b - a, n_types)), axis=1)[:, :LMAX]
        else:
            pick = rng.integers(0, n_types, size=(b - a, LMAX))
        E[a:b, : pick.shape[1]] = pick
        iv[a:b] = rng.integers(0, n_int, size=(b - a, LMAX - 1))
    pos = np.arange(LMAX)[None, :]
    E[pos >= L[:, None]] = 0
    iv[pos[:, : LMAX - 1] >= (L[:, None] - 1)] = 0
    return L, E, iv


def batched_recordings(seed=0xFE03, n_rec=256, t_range=(10.0, 600.0), m_range=(100, 20000),
                       lens=(2, 3, 4, 5, 6, 7, 8)):
    """Many recordings of uneven length with candidate sets of uneven size and length:
    per recording T log-uniform in t_range s, K uniform in 16..64, per-type rates uniform
    in [5, 50] Hz, 4 chains (lengths 4-6, 1-3 Hz, delays inside I_MS4 intervals); m
    log-uniform in m_range candidates with lengths drawn from `lens`; threshold 5x the
    chance count at the recording's mean rate and a 2 ms window."""
    rng = _rng(seed)
    recs = []
    for r in range(n_rec):
        T = float(np.exp(rng.uniform(np.log(t_range[0]), np.log(t_range[1]))))
        K = int(rng.integers(16, 65))
        rates = rng.uniform(5.0, 50.0, size=K)
        ch = _chains(rng, 4, K, [4, 5, 6], len(I_MS4), 1.0, 3.0)
        spec = [(tys, rate, [tuple(I_MS4[i]) for i in ivs]) for tys, ivs, rate in ch]
        t, ty = poisson_stream(seed * 1000 + r, K, rates, T, chains=spec)
        m = int(np.exp(rng.uniform(np.log(m_range[0]), np.log(m_range[1]))))
        cands = random_candidates(seed * 1000 + r + 500_000, m, K, list(lens), len(I_MS4))
        theta = chance_theta(float(rates.mean()), T, 0.002)
        recs.append(dict(stream=Stream(ty, t, K, ch), candidates=cands, theta=theta))
    return dict(name=f"batched_{n_rec}_recordings", recordings=recs, intervals=I_MS4.copy())


def level2_candidates(frequent_types, n_intervals):
    """All ordered pairs of distinct types, once per interval, in canonical order
    (first type, interval, second type)."""
    f = list(frequent_types)
    rows = [(a, iv, b) for a in f for iv in range(n_intervals) for b in f if a != b]
    m = len(rows)
    L = np.full(m, 2, np.uint8)
    E = np.zeros((m, LMAX), np.uint8)
    iv = np.zeros((m, LMAX - 1), np.uint8)
    for c, (a, i, b) in enumerate(rows):
        E[c, 0], E[c, 1], iv[c, 0] = a, b, i
    return L, E, iv


def tiny_stream(seed, n, n_types, max_gap_us, tie_prob=0.2):
    """A short random stream for brute-force checks: gaps uniform in [1, max_gap]
    with some zero gaps (timestamp ties)."""
    rng = _rng(seed)
    gaps = rng.integers(1, max_gap_us + 1, size=n)
    gaps[rng.random(n) < tie_prob] = 0
    t = np.cumsum(gaps).astype(np.uint32)
    ty = rng.integers(0, n_types, size=n).astype(np.uint8)
    return ty, t


def serving_streams(seed=0xFE05, n_streams=32, duration_s=90.0):
    """Simulated live recordings: per stream K uniform in 16..128 types, per-type rate
    uniform in [10, 100] Hz shared by the stream's types, 4 chains (lengths 4-6, 1-3 Hz,
    delays inside I_MS4 intervals)."""
    rng = _rng(seed)
    out = []
    for k in range(n_streams):
        K = int(rng.integers(16, 129))
        rate = float(rng.uniform(10.0, 100.0))
        ch = _chains(rng, 4, K, [4, 5, 6], len(I_MS4), 1.0, 3.0)
        spec = [(tys, r, [tuple(I_MS4[i]) for i in ivs]) for tys, ivs, r in ch]
        t, ty = poisson_stream(seed * 1000 + k, K, rate, duration_s, chains=spec)
        out.append(dict(stream=Stream(ty, t, K, ch), rate=rate))
    return out


def serving_requests(seed, rate_per_s, duration_s, n_streams, stream_types, m_range=(1000, 50000),
                     lens=(2, 3, 4, 5, 6), standing_frac=0.1):
    """Poisson request arrivals: (arrival s, stream, mode, candidate records seed, m)."""
    rng = _rng(seed)
    n = rng.poisson(rate_per_s * duration_s)
    arr = np.sort(rng.random(n) * duration_s)
    reqs = []
    for a in arr:
        sidx = int(rng.integers(0, n_streams))
        m = int(np.exp(rng.uniform(np.log(m_range[0]), np.log(m_range[1]))))
        standing = bool(rng.random() < standing_frac)
        reqs.append(dict(t=float(a), stream=sidx, m=m, standing=standing,
                         seed=int(rng.integers(0, 2**31)), K=stream_types[sidx], lens=lens))
    return reqs



def digest(*arrays) -> str:
    """SHA-256 over the bytes of the given arrays (shapes and dtypes included), so that
    a stored expected result can name the exact inputs it was computed from."""
    import hashlib
    h = hashlib.sha256()
    for a in arrays:
        a = np.ascontiguousarray(a)
        h.update(str((a.dtype.str, a.shape)).encode())
        h.update(a.tobytes())
    return h.hexdigest()
