"""Pins for the CPU oracle (no GPU).

Each check ties the oracle to something other than itself: the definition of
an occurrence and of the non-overlapped count (brute-force enumeration from
Section 2), hand-built worked streams that meet the paper's stated numbers
(tests/golden), closed forms, Theorem 5.1, anti-monotonicity, and, for the
exact MapConcatenate reference, the unsegmented count.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_0905_2200_gb300 import synth
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
pytestmark = pytest.mark.filterwarnings("ignore")


def load_golden(name):
    d = {"stream": [], "interval": []}
    section = None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            if parts[0] == "stream":
                section = "stream"
                continue
            if parts[0] in ("episode", "interval", "occurrences", "non_overlapped", "cut",
                            "serial_count", "naive_segment_sum", "tau", "exact_count",
                            "literal_count", "no_match", "several"):
                section = None
                vals = [int(x) for x in parts[1:]]
                if parts[0] == "interval":
                    d["interval"].append(vals)
                else:
                    d[parts[0]] = vals
                continue
            if section == "stream":
                d["stream"].append((int(parts[0]), int(parts[1])))
    ty = np.array([a for a, _ in d["stream"]], np.uint8)
    t = np.array([b for _, b in d["stream"]], np.uint32)
    lo = [iv[0] for iv in d["interval"]]
    hi = [iv[1] for iv in d["interval"]]
    return d, ty, t, d["episode"], lo, hi


def random_episode(rng, K, N, max_hi):
    E = [int(x) for x in rng.integers(0, K, size=N)]
    lo, hi = [], []
    for _ in range(N - 1):
        a = int(rng.integers(0, max_hi))
        b = int(rng.integers(a + 1, max_hi + 1))
        if rng.random() < 0.3:
            a = 0
        lo.append(a)
        hi.append(b)
    return E, lo, hi


# --------------------------------------------------------------------------- definition pins
@pytest.mark.parametrize("seed", range(60))
def test_exact_counts_equal_brute_force(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(0, 32))
    K = int(rng.integers(1, 5))
    ty, t = synth.tiny_stream(seed, n, K, 6, tie_prob=0.25)
    for _ in range(12):
        N = int(rng.integers(1, 5))
        E, lo, hi = random_episode(rng, K, N, 14)
        want = bf.count(ty, t, E, lo, hi)
        assert oracle.count_one(ty, t, E, lo, hi, oracle.EXACT) == want
        assert oracle.count_one(ty, t, E, lo, hi, oracle.EXACT_LISTS) == want


@pytest.mark.parametrize("seed", range(60))
def test_relaxed_counts_equal_brute_force(seed):
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(0, 32))
    K = int(rng.integers(1, 5))
    ty, t = synth.tiny_stream(seed + 500, n, K, 6, tie_prob=0.3)
    for _ in range(12):
        N = int(rng.integers(1, 5))
        E, lo, hi = random_episode(rng, K, N, 14)
        want = bf.count(ty, t, E, lo, hi, relaxed=True)
        assert oracle.count_one(ty, t, E, lo, hi, oracle.RELAXED) == want


@pytest.mark.parametrize("seed", range(40))
def test_greedy_equals_exhaustive_maximum(seed):
    """Earliest-end greedy (what Algorithm 1 realises) is a maximum non-overlapped set."""
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(1, 13))
    ty, t = synth.tiny_stream(seed + 900, n, 2, 4, tie_prob=0.2)
    for _ in range(6):
        E, lo, hi = random_episode(rng, 2, int(rng.integers(1, 4)), 8)
        for relaxed in (False, True):
            sp = bf.spans(bf.occurrences(ty, t, E, lo, hi, relaxed))
            assert bf.max_disjoint_greedy(sp) == bf.max_disjoint_exhaustive(sp)


def test_repeated_types_follow_descending_node_order():
    """A -> B -> A: the descending node loop lets one event serve two nodes of
    different partial occurrences; brute force agrees."""
    rng = np.random.default_rng(7)
    for s in range(40):
        ty, t = synth.tiny_stream(4000 + s, 28, 2, 5, tie_prob=0.2)
        for E in ([0, 1, 0], [0, 0], [1, 1, 1], [0, 0, 1]):
            lo = [0] * (len(E) - 1)
            hi = [int(x) for x in rng.integers(1, 12, size=len(E) - 1)]
            assert oracle.count_one(ty, t, E, lo, hi, oracle.EXACT) == bf.count(ty, t, E, lo, hi)
            assert oracle.count_one(ty, t, E, lo, hi, oracle.RELAXED) == bf.count(
                ty, t, E, lo, hi, relaxed=True)


# --------------------------------------------------------------------------- worked streams
def test_golden_fig2_eight_occurrences_two_non_overlapped():
    d, ty, t, E, lo, hi = load_golden("fig2_ab_occurrences.txt")
    occ = bf.occurrences(ty, t, E, lo, hi)
    assert len(occ) == d["occurrences"][0] == 8
    assert oracle.count_one(ty, t, E, lo, hi, oracle.EXACT) == d["non_overlapped"][1] == 2
    assert oracle.count_one(ty, t, E, lo, hi, oracle.EXACT_LISTS) == 2


def test_golden_fig2_one_constrained_occurrence():
    d, ty, t, E, lo, hi = load_golden("fig2_abc_constraints.txt")
    assert len(bf.occurrences(ty, t, E, lo, hi)) == d["occurrences"][0] == 1
    # several A..B..C triples exist in type order without the constraints
    assert len(bf.occurrences(ty, t, E, [0, 0], [10**6, 10**6])) > 1
    assert oracle.count_one(ty, t, E, lo, hi, oracle.EXACT) == 1
    assert oracle.count_one(ty, t, E, lo, hi, oracle.EXACT_LISTS) == 1


def test_golden_fig3_map_split_needs_boundary_state():
    d, ty, t, E, lo, hi = load_golden("fig3_map_split.txt")
    cut = d["cut"][0]
    serial = oracle.count_one(ty, t, E, lo, hi, oracle.EXACT)
    assert serial == d["serial_count"][0] == 3
    naive = (oracle.count_one(ty[:cut], t[:cut], E, lo, hi) +
             oracle.count_one(ty[cut:], t[cut:], E, lo, hi))
    assert naive == d["naive_segment_sum"][0] == 2
    assert oracle.count_mapconcat(ty, t, E, lo, hi, [0, cut, len(t)]) == serial


# --------------------------------------------------------------------------- closed forms
def test_single_node_count_is_type_histogram():
    ty, t = synth.tiny_stream(11, 500, 5, 3)
    hist = np.bincount(ty, minlength=5)
    for a in range(5):
        for p in (oracle.EXACT, oracle.EXACT_LISTS, oracle.RELAXED):
            assert oracle.count_one(ty, t, [a], [], [], p) == hist[a]


def test_planted_cascades_count_equals_triggers():
    """Noise-free cascades whose gaps exceed the episode span: every trigger is
    one occurrence and no two overlap."""
    rng = np.random.default_rng(5)
    E = [3, 1, 4, 0]
    lo, hi = [1000, 2000, 500], [2000, 4000, 1500]
    ty, t, cur = [], [], 0
    R = 57
    for _ in range(R):
        cur += 10_000 + int(rng.integers(0, 5000))
        x = cur
        for k, e in enumerate(E):
            if k:
                x += int(rng.integers(lo[k - 1] + 1, hi[k - 1] + 1))
            ty.append(e)
            t.append(x)
        cur = x
    ty, t = np.array(ty, np.uint8), np.array(t, np.uint32)
    for p in (oracle.EXACT, oracle.EXACT_LISTS, oracle.RELAXED):
        assert oracle.count_one(ty, t, E, lo, hi, p) == R
    # with distractor types interleaved the count is unchanged
    extra_t = np.sort(rng.integers(0, int(t[-1]), size=400)).astype(np.uint32)
    extra_ty = rng.integers(5, 9, size=400).astype(np.uint8)
    tt = np.concatenate([t, extra_t])
    yy = np.concatenate([ty, extra_ty])
    o = np.lexsort((yy, tt))
    assert oracle.count_one(yy[o], tt[o], E, lo, hi) == R


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_ordered_run_count_is_floor_run_over_n(N):
    """A run E1 E2 ... EN E1 E2 ... of R events, every delay inside its interval
    and every episode edge satisfied only by its own neighbours: floor(R / N)."""
    E = list(range(N))
    lo, hi = [100] * (N - 1), [200] * (N - 1)
    for R in range(0, 3 * N + 2):
        ty = np.array([E[k % N] for k in range(R)], np.uint8)
        t = (150 * np.arange(R)).astype(np.uint32)
        for p in (oracle.EXACT, oracle.EXACT_LISTS, oracle.RELAXED):
            assert oracle.count_one(ty, t, E, lo, hi, p) == R // N


def test_equal_times_never_chain_in_exact_pass_but_do_in_relaxed():
    ty = np.array([0, 1, 0, 1], np.uint8)
    t = np.array([10, 10, 20, 20], np.uint32)
    assert oracle.count_one(ty, t, [0, 1], [0], [5], oracle.EXACT) == 0
    assert oracle.count_one(ty, t, [0, 1], [0], [5], oracle.RELAXED) == 2


# --------------------------------------------------------------------------- invariants
@pytest.fixture(scope="module")
def tiny_cfg():
    return synth.tiny_mining()


def test_theorem_5_1_relaxed_bounds_exact(tiny_cfg):
    s = tiny_cfg["stream"]
    L, E, iv = synth.random_candidates(77, 600, 16, [2, 3, 4], 1)
    I = np.array([[4000, 6000]], np.uint32)
    ex = oracle.count_batch(s.types, s.t, L, E, iv, I, oracle.EXACT)
    rl = oracle.count_batch(s.types, s.t, L, E, iv, I, oracle.RELAXED)
    assert np.all(rl >= ex)
    assert np.any(rl > ex)


def test_exact_is_monotone_in_interval_width(tiny_cfg):
    s = tiny_cfg["stream"]
    rng = np.random.default_rng(3)
    for _ in range(40):
        N = int(rng.integers(2, 5))
        E = [int(x) for x in rng.choice(16, N, replace=False)]
        lo = [int(x) for x in rng.integers(0, 5000, N - 1)]
        hi = [a + int(x) for a, x in zip(lo, rng.integers(1, 8000, N - 1))]
        k = int(rng.integers(0, N - 1))
        lo2, hi2 = list(lo), list(hi)
        lo2[k] = max(0, lo2[k] - int(rng.integers(0, 2000)))
        hi2[k] = hi2[k] + int(rng.integers(0, 2000))
        assert (oracle.count_one(s.types, s.t, E, lo2, hi2) >=
                oracle.count_one(s.types, s.t, E, lo, hi))


def test_count_bounded_by_prefix_suffix_and_type_counts(tiny_cfg):
    s = tiny_cfg["stream"]
    hist = np.bincount(s.types, minlength=16)
    rng = np.random.default_rng(4)
    for _ in range(60):
        N = int(rng.integers(2, 5))
        E = [int(x) for x in rng.choice(16, N, replace=False)]
        lo = [int(x) for x in rng.integers(0, 4000, N - 1)]
        hi = [a + int(x) for a, x in zip(lo, rng.integers(1, 6000, N - 1))]
        for p in (oracle.EXACT, oracle.RELAXED):
            c = oracle.count_one(s.types, s.t, E, lo, hi, p)
            pre = oracle.count_one(s.types, s.t, E[:-1], lo[:-1], hi[:-1], p)
            suf = oracle.count_one(s.types, s.t, E[1:], lo[1:], hi[1:], p)
            assert c <= min(pre, suf)
            assert c <= min(hist[e] for e in E)


def test_pruned_lists_equal_literal_lists():
    """The windowed reading of Algorithm 1 (drop entries older than hi) equals the
    literal unpruned lists on a medium stream with many episodes."""
    s = synth.tiny_mining()["stream"]
    L, E, iv = synth.random_candidates(12, 300, 16, [2, 3, 4, 5], 3)
    I = np.array([[0, 3000], [4000, 6000], [1000, 9000]], np.uint32)
    a = oracle.count_batch(s.types, s.t, L, E, iv, I, oracle.EXACT)
    b = oracle.count_batch(s.types, s.t, L, E, iv, I, oracle.EXACT_LISTS)
    assert np.array_equal(a, b)


# --------------------------------------------------------------------------- MapConcatenate
def _random_bounds(rng, n, P, ty_t=None):
    if P >= n:
        return list(range(n + 1))
    cuts = sorted(rng.choice(np.arange(1, n), size=P - 1, replace=False).tolist())
    return [0] + cuts + [n]


@pytest.mark.parametrize("seed", range(25))
def test_mapconcat_equals_unsegmented_tiny(seed):
    rng = np.random.default_rng(5000 + seed)
    n = int(rng.integers(1, 40))
    K = int(rng.integers(1, 4))
    ty, t = synth.tiny_stream(6000 + seed, n, K, 4, tie_prob=0.3)
    for _ in range(8):
        N = int(rng.integers(1, 5))
        E, lo, hi = random_episode(rng, K, N, 10)
        for p in (oracle.EXACT, oracle.RELAXED):
            want = oracle.count_one(ty, t, E, lo, hi, p)
            for P in (1, 2, 3, max(1, n // 2), n):
                b = _random_bounds(rng, n, P)
                assert oracle.count_mapconcat(ty, t, E, lo, hi, b, p) == want


def test_mapconcat_equals_unsegmented_medium_many_segments():
    cfg = synth.tiny_mining()
    s = cfg["stream"]
    rng = np.random.default_rng(9)
    L, E, iv = synth.random_candidates(21, 40, 16, [2, 3, 4], 1)
    I = np.array([[4000, 6000]], np.uint32)
    lo_all, hi_all = oracle.resolve(L, E, iv, I)
    n = s.n
    for c in range(len(L)):
        N = int(L[c])
        Ec, lo, hi = list(E[c, :N]), list(lo_all[c, : N - 1]), list(hi_all[c, : N - 1])
        for p in (oracle.EXACT, oracle.RELAXED):
            want = oracle.count_one(s.types, s.t, Ec, lo, hi, p)
            for P in (7, 64, 1000):
                b = _random_bounds(rng, n, P)
                assert oracle.count_mapconcat(s.types, s.t, Ec, lo, hi, b, p) == want


def test_mapconcat_cuts_at_timestamp_ties():
    ty, t = synth.tiny_stream(77, 200, 3, 2, tie_prob=0.6)
    ties = [j for j in range(1, len(t)) if t[j] == t[j - 1]]
    assert len(ties) > 20
    rng = np.random.default_rng(1)
    for _ in range(30):
        E, lo, hi = random_episode(rng, 3, int(rng.integers(2, 5)), 6)
        b = [0] + sorted(rng.choice(ties, size=10, replace=False).tolist()) + [len(t)]
        for p in (oracle.EXACT, oracle.RELAXED):
            assert (oracle.count_mapconcat(ty, t, E, lo, hi, b, p) ==
                    oracle.count_one(ty, t, E, lo, hi, p))


# --------------------------------------------------------------------------- miner
def _bf_mine(ty, t, K, I, theta, max_len, repeated_types=False):
    """Every episode up to max_len (distinct-type unless repeated_types), counted by
    brute force (maximum non-overlapped set of enumerated occurrences), kept if >= theta."""
    hist = np.bincount(ty, minlength=K)
    res = {1: [((a,), (), int(hist[a])) for a in range(K) if hist[a] >= theta]}
    eps = list(bf.all_episodes(K, len(I), max_len, repeated_types))
    if repeated_types:
        cnt = [bf.count(ty, t, list(tys), [int(I[i][0]) for i in ivs], [int(I[i][1]) for i in ivs])
               for tys, ivs in eps]
    else:
        lens, E, iv = oracle._pack(eps)
        cnt = oracle.count_batch(ty, t, lens, E, iv, I, oracle.EXACT)
    for (tys, ivs), c in zip(eps, cnt):
        if c >= theta:
            res.setdefault(len(tys), []).append((tys, ivs, int(c)))
    for k in res:
        res[k].sort(key=lambda r: oracle.canonical_key(r[0], r[1]))
    return res


@pytest.mark.parametrize("seed", range(8))
def test_levelwise_miner_equals_brute_force_miner(seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(2, 5))
    nI = int(rng.integers(1, 3))
    chain = tuple(int(x) for x in rng.choice(K, size=min(K, 3), replace=False))
    t, ty = synth.poisson_stream(700 + seed, K, 8.0, 20.0,
                                 chains=[(chain, 3.0, [(2000, 6000)] * (len(chain) - 1))])
    I = np.array([[2000, 6000], [0, 3000]][:nI], np.uint32)
    theta = int(rng.integers(8, 30))
    got = oracle.mine(ty, t, K, I, theta, 4)
    want = _bf_mine(ty, t, K, I, theta, 4)
    assert got == {k: v for k, v in want.items() if v}
    assert len(got) >= 2


@pytest.mark.parametrize("seed", range(4))
def test_repeated_type_miner_equals_brute_force_miner(seed):
    """Mining with repeated types allowed (A -> B -> A): every episode over 2-3 types
    up to length 3 counted by brute force (occurrence enumeration + maximum
    non-overlapped set), against the level-wise miner with the repeat-keeping join."""
    rng = np.random.default_rng(40 + seed)
    K = int(rng.integers(2, 4))
    t, ty = synth.poisson_stream(800 + seed, K, 4.0, 6.0,
                                 chains=[((0, 1, 0), 3.0, [(2000, 6000)] * 2)])
    I = np.array([[2000, 6000], [0, 3000]], np.uint32)
    theta = int(rng.integers(6, 10))
    got = oracle.mine(ty, t, K, I, theta, 3, repeated_types=True)
    want = _bf_mine(ty, t, K, I, theta, 3, repeated_types=True)
    assert got == {k: v for k, v in want.items() if v}
    assert any(len(set(r[0])) < len(r[0]) for lv in got.values() for r in lv)


def test_two_pass_miner_equals_exact_only_miner():
    cfg = synth.tiny_mining()
    s = cfg["stream"]
    a = oracle.mine(s.types, s.t, 16, cfg["intervals"], cfg["theta"], cfg["max_len"], True)
    b = oracle.mine(s.types, s.t, 16, cfg["intervals"], cfg["theta"], cfg["max_len"], False)
    assert a == b
    # the embedded cascade 0 -> 1 -> 2 -> 3 is found at full length
    assert any(r[0] == (0, 1, 2, 3) for r in a.get(4, []))


def test_join_output_is_canonical_and_distinct_typed():
    freq = [((0, 1), (0,)), ((1, 2), (0,)), ((1, 2), (1,)), ((1, 0), (1,)), ((2, 3), (0,))]
    out = oracle.join(freq)
    assert out == [((0, 1, 2), (0, 0)), ((0, 1, 2), (0, 1)),
                   ((1, 2, 3), (0, 0)), ((1, 2, 3), (1, 0))]
    keys = [oracle.canonical_key(*c) for c in out]
    assert keys == sorted(keys)


# --------------------------------------------------------------------------- MapConcatenate as printed
@pytest.mark.parametrize("seed", range(30))
def test_literal_mapconcat_single_segment_is_algorithm_1(seed):
    """With one time segment the printed scheme is one machine over the whole stream."""
    rng = np.random.default_rng(9000 + seed)
    ty, t = synth.tiny_stream(9000 + seed, int(rng.integers(1, 40)), 3, 5, tie_prob=0.25)
    E, lo, hi = random_episode(rng, 3, int(rng.integers(1, 4)), 8)
    got = oracle.count_mapconcat_literal(ty, t, E, lo, hi, [int(t[0]) - 1, int(t[-1])])[0]
    assert got == bf.count(ty, t, E, lo, hi)


def test_literal_mapconcat_fig3_recovers_the_serial_count():
    """Fig. 3's stream: a fresh machine on the second segment finds g and misses h3;
    the printed scheme's machine started W earlier does not, so the count is the
    serial one (3), where summing fresh per-segment machines gives 2."""
    d, ty, t, E, lo, hi = load_golden("fig3_map_split.txt")
    cut = d["cut"][0]
    tau = [int(t[0]) - 1, int(t[cut - 1]), int(t[-1])]
    got, tup, diag = oracle.count_mapconcat_literal(ty, t, E, lo, hi, tau)
    assert got == d["serial_count"][0] == 3
    assert tup[1, 0, 1] + tup[0, 0, 1] == d["naive_segment_sum"][0]   # machine 0 alone
    assert tup[0, 0, 2] == tup[1, 1, 0]                              # b of seg 0 = a of machine 1


@pytest.mark.parametrize("name", ["literal_mc_d1_short_segments.txt",
                                  "literal_mc_d2_window_edge.txt",
                                  "literal_mc_d3_machine_out_of_step.txt"])
def test_literal_mapconcat_catalogued_divergences(name):
    """Three hand-traced streams on which the printed scheme undercounts (the exact
    reformulation does not): D1 occurrences spanning more than two segments, D2 an
    occurrence ending exactly at tau + W, D3 machines out of step with the serial
    machine's last completion."""
    d, ty, t, E, lo, hi = load_golden(name)
    got, tup, diag = oracle.count_mapconcat_literal(ty, t, E, lo, hi, d["tau"])
    assert oracle.count_one(ty, t, E, lo, hi, oracle.EXACT) == bf.count(ty, t, E, lo, hi) \
        == d["exact_count"][0]
    assert got == d["literal_count"][0]
    assert diag == (d["no_match"][0], d["several"][0])
    # the exact reformulation over the same cut points (index ranges) is exact
    idx = [0] + [int(np.searchsorted(t, x, side="right")) for x in d["tau"][1:-1]] + [len(t)]
    idx = sorted(set(idx))
    assert oracle.count_mapconcat(ty, t, E, lo, hi, idx) == d["exact_count"][0]


# --------------------------------------------------------------------------- window-based frequency
@pytest.mark.parametrize("seed", range(40))
def test_window_count_equals_brute_force(seed):
    """The window-based frequency (Section 2's alternative measure) by the oracle's
    recurrence over nodes equals the union of every occurrence's window starts."""
    rng = np.random.default_rng(6000 + seed)
    ty, t = synth.tiny_stream(6000 + seed, int(rng.integers(1, 30)), 3, 4, tie_prob=0.2)
    E, lo, hi = random_episode(rng, 3, int(rng.integers(1, 4)), 8)
    for w in (1, 3, 9, 30):
        assert oracle.count_windows(ty, t, E, lo, hi, w) == bf.window_count(ty, t, E, lo, hi, w)


def test_window_count_single_node_and_empty():
    """One node: each event covers w starts, merged where they overlap; an episode
    that never occurs covers none."""
    ty = np.array([0, 0, 1, 0], np.uint8)
    t = np.array([10, 12, 13, 40], np.uint32)
    assert oracle.count_windows(ty, t, [0], [], [], 5) == len(set(range(6, 11)) | set(range(8, 13))
                                                              | set(range(36, 41)))
    assert oracle.count_windows(ty, t, [1, 1], [0], [5], 5) == 0
