"""Plain CPU oracle for frequent-episode counting and mining (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of the
benchmark may import this package.  The product library never imports, links
or calls it, and this package never imports the product library: the two share
no code.  Inputs come from the seeded generators (which hold none of the
method's arithmetic) or from hand-written fixtures.

Contents
--------
``fem_oracle.c`` (compiled with gcc by :func:`build`) holds the counters:
Algorithm 1 literal (unpruned lists), Algorithm 1 with pruned lists,
Algorithm 3, Algorithm 4 and the exact MapConcatenate reference.  This module
wraps them and adds the level-wise miner (Problem 1, Section 2; level-wise
candidate generation as the paper's Section 5 introduction describes it),
written as plain Python over the C counters.

Episode encoding used by every function here: ``len`` (uint8[m]),
``types`` (uint8[m, 8], unused tail ignored) and ``ivl`` (uint8[m, 7], indices
into the interval table ``intervals`` = uint32[nI, 2] of (lo, hi] pairs in
microseconds).  Parity for the paper's own figures is unpinned: the figures
are missing from the source text.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

LMAX = 8
RELAXED, EXACT, EXACT_LISTS = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fem_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libfem_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``fem_oracle.c`` into ``oracle/_build/libfem_oracle.so``."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        # FEM_ORACLE_LIB names another build of fem_oracle.c: the mutation tests load
        # copies with a planted mistake through it, to show the pins catch them
        lib = ctypes.CDLL(os.environ.get("FEM_ORACLE_LIB") or build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i64 = ctypes.c_int64
        lib.orc_count_exact_lists.restype = ctypes.c_uint32
        lib.orc_count_exact_lists.argtypes = [u8p, u32p, i64, ctypes.c_int, u8p, u32p, u32p]
        lib.orc_count_exact.restype = ctypes.c_uint32
        lib.orc_count_exact.argtypes = [u8p, u32p, i64, ctypes.c_int, u8p, u32p, u32p]
        lib.orc_count_relaxed.restype = ctypes.c_uint32
        lib.orc_count_relaxed.argtypes = [u8p, u32p, i64, ctypes.c_int, u8p, u32p]
        lib.orc_count_batch.restype = ctypes.c_int
        lib.orc_count_batch.argtypes = [u8p, u32p, i64, i64, u8p, u8p, u32p, u32p,
                                        ctypes.c_int, u32p]
        lib.orc_two_pass.restype = ctypes.c_int
        lib.orc_two_pass.argtypes = [u8p, u32p, i64, i64, u8p, u8p, u32p, u32p,
                                     ctypes.c_uint32, u32p, u32p, u8p]
        lib.orc_count_windows.restype = ctypes.c_uint64
        lib.orc_count_windows.argtypes = [u8p, u32p, i64, ctypes.c_int, u8p, u32p, u32p,
                                          ctypes.c_uint32]
        lib.orc_count_mapconcat_literal.restype = ctypes.c_uint32
        lib.orc_count_mapconcat_literal.argtypes = [u8p, u32p, i64, ctypes.c_int, u8p, u32p,
                                                    u32p, i64, i64p, i64p, i64p]
        lib.orc_count_mapconcat.restype = ctypes.c_uint32
        lib.orc_count_mapconcat.argtypes = [u8p, u32p, i64, ctypes.c_int, u8p, u32p, u32p,
                                            ctypes.c_int, i64, i64p, i64p]
        _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _stream(types, t):
    types = np.ascontiguousarray(types, dtype=np.uint8)
    t = np.ascontiguousarray(t, dtype=np.uint32)
    if types.shape != t.shape:
        raise ValueError("types and t differ in length")
    return types, t


def _edges(ep_types, lo, hi):
    E = np.zeros(LMAX, np.uint8)
    E[: len(ep_types)] = ep_types
    L = np.zeros(LMAX - 1, np.uint32)
    H = np.zeros(LMAX - 1, np.uint32)
    L[: len(lo)] = lo
    H[: len(hi)] = hi
    return E, L, H


# --------------------------------------------------------------------------- single episodes
def count_one(types, t, ep_types, lo, hi, pass_=EXACT) -> int:
    """Count one episode given explicit per-edge (lo, hi] bounds."""
    lib = _load()
    types, t = _stream(types, t)
    N = len(ep_types)
    if not 1 <= N <= LMAX or len(lo) != N - 1 or len(hi) != N - 1:
        raise ValueError("bad episode")
    E, L, H = _edges(ep_types, lo, hi)
    n = len(t)
    if pass_ == RELAXED:
        r = lib.orc_count_relaxed(_p(types, ctypes.c_uint8), _p(t, ctypes.c_uint32), n, N,
                                  _p(E, ctypes.c_uint8), _p(H, ctypes.c_uint32))
    elif pass_ == EXACT:
        r = lib.orc_count_exact(_p(types, ctypes.c_uint8), _p(t, ctypes.c_uint32), n, N,
                                _p(E, ctypes.c_uint8), _p(L, ctypes.c_uint32),
                                _p(H, ctypes.c_uint32))
    elif pass_ == EXACT_LISTS:
        r = lib.orc_count_exact_lists(_p(types, ctypes.c_uint8), _p(t, ctypes.c_uint32), n, N,
                                      _p(E, ctypes.c_uint8), _p(L, ctypes.c_uint32),
                                      _p(H, ctypes.c_uint32))
    else:
        raise ValueError("bad pass")
    if r == 0xFFFFFFFF:
        raise MemoryError("oracle ran out of memory")
    return int(r)


def count_mapconcat(types, t, ep_types, lo, hi, bounds, pass_=EXACT, return_sizes=False):
    """Exact MapConcatenate count over the index segmentation ``bounds``."""
    lib = _load()
    types, t = _stream(types, t)
    N = len(ep_types)
    E, L, H = _edges(ep_types, lo, hi)
    b = np.ascontiguousarray(bounds, dtype=np.int64)
    P = len(b) - 1
    sizes = np.zeros(max(P, 1), np.int64)
    r = lib.orc_count_mapconcat(_p(types, ctypes.c_uint8), _p(t, ctypes.c_uint32), len(t), N,
                                _p(E, ctypes.c_uint8), _p(L, ctypes.c_uint32),
                                _p(H, ctypes.c_uint32), 1 if pass_ != RELAXED else 0, P,
                                _p(b, ctypes.c_int64), _p(sizes, ctypes.c_int64))
    if r == 0xFFFFFFFF:
        raise ValueError("bad segmentation or out of memory")
    return (int(r), sizes[:P]) if return_sizes else int(r)


def capacity_table(types, t, n_types, widths):
    """cap[a, j]: the most events of type a inside one closed window of length widths[j]
    (microseconds), max over x of #{i : types[i] = a, x <= t[i] <= x + widths[j]}.

    It bounds the state of the counters: Algorithm 1's list for node k keeps, once the
    entries older than hi_k are dropped, events of type E_k within hi_k of the newest
    one, so at most cap[E_k, hi_k] of them (Section 5.1); a MapConcatenate segment
    (Section 5.2.2) tabulates one entry class per last-node event in its look-back
    window of length W = sum of hi, so at most 1 + cap[E_N, W] classes.  A fullest
    window can be moved to start at one of its events, so counting forward from each
    event of the type is enough (a sorted search over the type's times)."""
    types, t = _stream(types, t)
    widths = np.asarray(widths, dtype=np.uint64).reshape(-1)
    cap = np.zeros((n_types, len(widths)), np.uint32)
    for a in range(n_types):
        ts = t[types == a].astype(np.uint64)
        if len(ts) == 0:
            continue
        first = np.arange(len(ts))
        for j, h in enumerate(widths):
            last = np.searchsorted(ts, ts + h, side="right")
            cap[a, j] = int((last - first).max())
    return cap


def count_windows(types, t, ep_types, lo, hi, w):
    """Window-based frequency (Section 2's alternative measure, with the episode's
    interval constraints): how many integer starts s have an occurrence inside the
    window [s, s + w)."""
    lib = _load()
    types, t = _stream(types, t)
    N = len(ep_types)
    E, L, H = _edges(ep_types, lo, hi)
    r = lib.orc_count_windows(_p(types, ctypes.c_uint8), _p(t, ctypes.c_uint32), len(t), N,
                              _p(E, ctypes.c_uint8), _p(L, ctypes.c_uint32),
                              _p(H, ctypes.c_uint32), int(w))
    if r == 0xFFFFFFFFFFFFFFFF:
        raise ValueError("bad episode or window, or out of memory")
    return int(r)


def count_windows_batch(types, t, lens, ep_types, ivl, intervals, w):
    """count_windows for m candidates given as (len, types, interval indices)."""
    lo, hi = resolve(lens, ep_types, ivl, intervals)
    E = np.asarray(ep_types, dtype=np.uint8).reshape(-1, LMAX)
    return np.array([count_windows(types, t, E[i, :int(lens[i])], lo[i, :int(lens[i]) - 1],
                                   hi[i, :int(lens[i]) - 1], w) for i in range(len(lens))],
                    np.uint64)


def count_mapconcat_literal(types, t, ep_types, lo, hi, tau):
    """MapConcatenate as the paper prints it (Section 5.2.2; readings in fem_oracle.c):
    time segments (tau[p], tau[p+1]], N machines per segment, tuples (a, count, b)
    joined where b equals a.  Returns (count, tuples int64[P, N, 3], diag) where diag =
    (boundaries where no tuple matched, boundaries where several did)."""
    lib = _load()
    types, t = _stream(types, t)
    N = len(ep_types)
    E, L, H = _edges(ep_types, lo, hi)
    tau = np.ascontiguousarray(tau, dtype=np.int64)
    P = len(tau) - 1
    tup = np.zeros((max(P, 1), N, 3), np.int64)
    diag = np.zeros(2, np.int64)
    r = lib.orc_count_mapconcat_literal(_p(types, ctypes.c_uint8), _p(t, ctypes.c_uint32),
                                        len(t), N, _p(E, ctypes.c_uint8), _p(L, ctypes.c_uint32),
                                        _p(H, ctypes.c_uint32), P, _p(tau, ctypes.c_int64),
                                        _p(tup, ctypes.c_int64), _p(diag, ctypes.c_int64))
    if r == 0xFFFFFFFF:
        raise ValueError("bad time segmentation or out of memory")
    return int(r), tup[:P], (int(diag[0]), int(diag[1]))


# --------------------------------------------------------------------------- candidate batches
def resolve(lens, ep_types, ivl, intervals):
    """Turn interval indices into per-edge lo/hi arrays (uint32[m, 7] each)."""
    intervals = np.asarray(intervals, dtype=np.uint32).reshape(-1, 2)
    ivl = np.asarray(ivl, dtype=np.int64).reshape(-1, LMAX - 1)
    lens = np.asarray(lens, dtype=np.int64)
    m = len(lens)
    lo = np.zeros((m, LMAX - 1), np.uint32)
    hi = np.zeros((m, LMAX - 1), np.uint32)
    for k in range(LMAX - 1):
        on = lens > k + 1
        lo[on, k] = intervals[ivl[on, k], 0]
        hi[on, k] = intervals[ivl[on, k], 1]
    return lo, hi


def count_batch(types, t, lens, ep_types, ivl, intervals, pass_=EXACT) -> np.ndarray:
    """Count m candidates one after the other; returns uint32[m]."""
    lib = _load()
    types, t = _stream(types, t)
    lens = np.ascontiguousarray(lens, dtype=np.uint8)
    E = np.ascontiguousarray(np.asarray(ep_types, dtype=np.uint8).reshape(-1, LMAX))
    lo, hi = resolve(lens, E, ivl, intervals)
    out = np.zeros(len(lens), np.uint32)
    rc = lib.orc_count_batch(_p(types, ctypes.c_uint8), _p(t, ctypes.c_uint32), len(t),
                             len(lens), _p(lens, ctypes.c_uint8), _p(E, ctypes.c_uint8),
                             _p(lo, ctypes.c_uint32), _p(hi, ctypes.c_uint32), pass_,
                             _p(out, ctypes.c_uint32))
    if rc:
        raise ValueError(f"oracle count_batch failed ({rc})")
    return out


def two_pass(types, t, lens, ep_types, ivl, intervals, theta):
    """Algorithm 4: returns (relaxed uint32[m], exact-or-zero uint32[m], survived uint8[m])."""
    lib = _load()
    types, t = _stream(types, t)
    lens = np.ascontiguousarray(lens, dtype=np.uint8)
    E = np.ascontiguousarray(np.asarray(ep_types, dtype=np.uint8).reshape(-1, LMAX))
    lo, hi = resolve(lens, E, ivl, intervals)
    m = len(lens)
    rel = np.zeros(m, np.uint32)
    ex = np.zeros(m, np.uint32)
    sv = np.zeros(m, np.uint8)
    rc = lib.orc_two_pass(_p(types, ctypes.c_uint8), _p(t, ctypes.c_uint32), len(t), m,
                          _p(lens, ctypes.c_uint8), _p(E, ctypes.c_uint8),
                          _p(lo, ctypes.c_uint32), _p(hi, ctypes.c_uint32), int(theta),
                          _p(rel, ctypes.c_uint32), _p(ex, ctypes.c_uint32),
                          _p(sv, ctypes.c_uint8))
    if rc:
        raise ValueError(f"oracle two_pass failed ({rc})")
    return rel, ex, sv


# --------------------------------------------------------------------------- level-wise miner
def canonical_key(ep_types, ivl):
    """Interleaved key (E1, iv1, E2, iv2, ..., E_N): the order results are listed in."""
    key = []
    for k, e in enumerate(ep_types):
        key.append(int(e))
        if k < len(ivl):
            key.append(int(ivl[k]))
    return tuple(key)


def _pack(cands):
    m = len(cands)
    lens = np.zeros(m, np.uint8)
    E = np.zeros((m, LMAX), np.uint8)
    iv = np.zeros((m, LMAX - 1), np.uint8)
    for c, (ty, ix) in enumerate(cands):
        lens[c] = len(ty)
        E[c, : len(ty)] = ty
        iv[c, : len(ix)] = ix
    return lens, E, iv


def join(frequent, repeated_types=False):
    """Next-level candidates from the frequent N-node episodes.

    alpha and beta join when alpha without its first node equals beta without
    its last node (types and intervals); the candidate is alpha followed by
    beta's last edge and node, kept only if that node's type is new to alpha
    (episodes are tuples of distinct types, Def. 2.2) unless ``repeated_types``
    (then every such candidate is kept: dropping the first or last node of an
    episode with repeated types cannot lower its count either).  Returned in
    canonical order.
    """
    by_prefix = {}
    for ty, ix in frequent:
        by_prefix.setdefault((ty[:-1], ix[:-1]), []).append((ty, ix))
    out = []
    for ty, ix in frequent:
        for bty, bix in by_prefix.get((ty[1:], ix[1:]), []):
            if bty[-1] in ty and not repeated_types:
                continue
            out.append((ty + (bty[-1],), ix + (bix[-1],)))
    out.sort(key=lambda c: canonical_key(*c))
    return out


def mine(types, t, n_types, intervals, theta, max_len, two_pass_counting=True,
         repeated_types=False, counter=None):
    """Problem 1 (Section 2), level by level.

    Level 1: the count of a one-node episode is the number of events of its
    type.  Level 2: every ordered pair of distinct frequent types, once per
    interval.  Level N+1: :func:`join` of level N's frequent set.  Each level is
    counted with Algorithm 4 (relaxed pass, drop below theta, exact pass) or,
    if ``two_pass_counting`` is False, with the exact pass alone.  An episode is
    frequent iff its exact count is >= theta.  With ``repeated_types`` a type may
    appear at several nodes (level 2 includes (a, a); the join keeps repeats).

    ``counter``: an object with ``two_pass`` and ``count_batch`` methods taking
    the arguments of the module functions minus the stream (``oracle.shards.
    ShardPool``, the same counters run over candidate shards); None counts here.

    Returns {level: [(types tuple, interval-index tuple, count), ...]} with
    each level in canonical order; level 1 lists (type,), (), count.
    """
    types, t = _stream(types, t)
    intervals = np.asarray(intervals, dtype=np.uint32).reshape(-1, 2)
    hist = np.bincount(types, minlength=n_types)
    res = {1: [((a,), (), int(hist[a])) for a in range(n_types) if hist[a] >= theta]}
    f1 = [a for a in range(n_types) if hist[a] >= theta]
    cands = [((a, b), (iv,)) for a in f1 for iv in range(len(intervals)) for b in f1
             if a != b or repeated_types]
    level = 2
    while cands and level <= max_len:
        lens, E, iv = _pack(cands)
        if two_pass_counting:
            if counter is None:
                _, exact, sv = two_pass(types, t, lens, E, iv, intervals, theta)
            else:
                _, exact, sv = counter.two_pass(lens, E, iv, intervals, theta)
            keep = (sv != 0) & (exact >= theta)
        else:
            if counter is None:
                exact = count_batch(types, t, lens, E, iv, intervals, EXACT)
            else:
                exact = counter.count_batch(lens, E, iv, intervals, EXACT)
            keep = exact >= theta
        freq = [(cands[c][0], cands[c][1], int(exact[c])) for c in range(len(cands)) if keep[c]]
        if not freq:
            break
        res[level] = freq
        if level == max_len:
            break
        cands = join([(ty, ix) for ty, ix, _ in freq], repeated_types)
        level += 1
    return res
