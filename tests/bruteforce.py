"""Brute-force definitions used to pin the oracle (pure Python, tiny inputs only).

Nothing here is shared with the oracle: occurrences are enumerated straight
from the definition in Section 2 of the paper (an occurrence maps the N nodes
to events i_1 < ... < i_N of the right types whose consecutive delays lie in
the edges' intervals), and the largest non-overlapped set is found two ways
(earliest-end greedy, and an exhaustive search) so that each checks the other.
"""
from __future__ import annotations

import functools
import itertools


def occurrences(types, t, E, lo, hi, relaxed=False):
    """All occurrences of the episode (E; (lo, hi] per edge) as index tuples.

    relaxed=True uses 0 <= delay <= hi for every edge (the lower bounds dropped
    and zero delays allowed, the relaxed episode of Section 5.3.1)."""
    n = len(t)
    N = len(E)
    pos = [[j for j in range(n) if int(types[j]) == int(E[k])] for k in range(N)]
    out = []

    def rec(k, acc):
        if k == N:
            out.append(tuple(acc))
            return
        for j in pos[k]:
            if acc:
                p = acc[-1]
                if j <= p:
                    continue
                d = int(t[j]) - int(t[p])
                ok = (0 <= d <= int(hi[k - 1])) if relaxed else (int(lo[k - 1]) < d <= int(hi[k - 1]))
                if not ok:
                    continue
            acc.append(j)
            rec(k + 1, acc)
            acc.pop()

    rec(0, [])
    return out


def spans(occs):
    return sorted({(o[0], o[-1]) for o in occs})


def max_disjoint_greedy(sp):
    """Earliest-end greedy interval scheduling over closed index spans."""
    count, last = 0, -1
    for s, e in sorted(sp, key=lambda x: (x[1], x[0])):
        if s > last:
            count += 1
            last = e
    return count


def max_disjoint_exhaustive(sp):
    """Largest set of pairwise disjoint spans by trying every take/skip choice
    (memoised on the position and the last taken end)."""
    sp = sorted(sp)

    @functools.lru_cache(maxsize=None)
    def best(i, last):
        if i == len(sp):
            return 0
        s, e = sp[i]
        skip = best(i + 1, last)
        take = 1 + best(i + 1, e) if s > last else 0
        return max(skip, take)

    return best(0, -1)


def count(types, t, E, lo, hi, relaxed=False):
    return max_disjoint_greedy(spans(occurrences(types, t, E, lo, hi, relaxed)))


def all_episodes(n_types, n_intervals, max_len, repeated_types=False):
    """Every episode of 2..max_len nodes, distinct-type unless repeated_types:
    (types tuple, interval-index tuple)."""
    for N in range(2, max_len + 1):
        tuples = (itertools.product(range(n_types), repeat=N) if repeated_types
                  else itertools.permutations(range(n_types), N))
        for tys in tuples:
            for ivs in itertools.product(range(n_intervals), repeat=N - 1):
                yield tys, ivs


def window_count(types, t, E, lo, hi, w):
    """Number of integer window starts s such that some occurrence lies inside
    [s, s + w): the union over occurrences of the starts in (t_last - w, t_first]."""
    starts = set()
    for o in occurrences(types, t, E, lo, hi):
        a, b = int(t[o[-1]]) - w + 1, int(t[o[0]])
        starts.update(range(a, b + 1))
    return len(starts)
