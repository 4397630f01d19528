"""The oracle's plain counters run as independent processes over candidate shards.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the tests, the golden-file
writer beside this module and the benchmark's CPU-baseline leg use it.

Nothing here changes what is computed.  Each worker process loads the same
single-threaded C oracle (``fem_oracle.c``) and runs :func:`oracle.two_pass` or
:func:`oracle.count_batch` on a contiguous slice of the candidates; the slices'
results are concatenated in order.  Counts of different episodes are independent
(each episode runs its own machine over the whole stream, Algorithms 1 and 3), so
the sharded result is the single-process result.  The pool is started with the
``spawn`` method, so it is safe in a process that has already used a GPU.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from . import EXACT, count_batch, two_pass

_S = {}


def _init(types, t):
    _S["types"] = types
    _S["t"] = t


def _two_pass(args):
    L, E, iv, intervals, theta = args
    return two_pass(_S["types"], _S["t"], L, E, iv, intervals, theta)


def _two_pass_stream(args):
    types, t, L, E, iv, intervals, theta = args
    return two_pass(types, t, L, E, iv, intervals, theta)


def two_pass_jobs(jobs, procs: int | None = None):
    """Algorithm 4 for many (types, t, L, E, iv, intervals, theta) jobs, each on its own
    stream, spread over ``procs`` spawned processes; results in job order."""
    procs = int(procs or os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_two_pass_stream, list(jobs), chunksize=1)


def _count(args):
    L, E, iv, intervals, pass_ = args
    return count_batch(_S["types"], _S["t"], L, E, iv, intervals, pass_)


def _slices(m, parts):
    parts = max(1, min(parts, m))
    edges = np.linspace(0, m, parts + 1).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


class ShardPool:
    """``procs`` worker processes (default: every host core) holding one stream.

    Use as a context manager.  :meth:`two_pass` and :meth:`count_batch` have the
    signatures of the module functions minus the stream arguments."""

    def __init__(self, types, t, procs: int | None = None):
        self.procs = int(procs or os.cpu_count() or 1)
        types = np.ascontiguousarray(types, dtype=np.uint8)
        t = np.ascontiguousarray(t, dtype=np.uint32)
        self._pool = mp.get_context("spawn").Pool(self.procs, initializer=_init,
                                                  initargs=(types, t))
        self._memo = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def close(self):
        if self._pool is not None:
            self._pool.close()
            self._pool.join()
            self._pool = None

    def _parts(self, m):
        # several slices per process so that uneven episodes even out
        return _slices(m, 4 * self.procs)

    def two_pass(self, L, E, iv, intervals, theta):
        """Algorithm 4 over the shards; a repeated call with the same inputs returns the
        first call's arrays (the golden writer asks for one level twice)."""
        key = (np.asarray(L).tobytes(), np.asarray(E).tobytes(), np.asarray(iv).tobytes(),
               np.asarray(intervals).tobytes(), int(theta))
        if key not in self._memo:
            self._memo[key] = self._two_pass(L, E, iv, intervals, theta)
        return self._memo[key]

    def _two_pass(self, L, E, iv, intervals, theta):
        m = len(L)
        if m == 0:
            z = np.zeros(0, np.uint32)
            return z, z.copy(), np.zeros(0, np.uint8)
        E = np.asarray(E).reshape(m, -1)
        iv = np.asarray(iv).reshape(m, -1)
        jobs = [(L[a:b], E[a:b], iv[a:b], intervals, theta) for a, b in self._parts(m)]
        out = self._pool.map(_two_pass, jobs)
        return tuple(np.concatenate([o[k] for o in out]) for k in range(3))

    def count_batch(self, L, E, iv, intervals, pass_=EXACT):
        m = len(L)
        if m == 0:
            return np.zeros(0, np.uint32)
        E = np.asarray(E).reshape(m, -1)
        iv = np.asarray(iv).reshape(m, -1)
        jobs = [(L[a:b], E[a:b], iv[a:b], intervals, pass_) for a, b in self._parts(m)]
        return np.concatenate(self._pool.map(_count, jobs))
