"""Pins for the oracle's capacity table (no GPU): cap[a, h] is the most type-a events in
one closed window of length h.  Checked against a scan over every integer window start,
against its closed forms at h = 0 and at the stream's span, and against the quantity it
bounds: the entry classes of the exact MapConcatenate tables (Section 5.2.2), one per
last-node event of a look-back window of length W = sum of hi."""
import numpy as np
import pytest

import oracle
from paper_0905_2200_gb300 import synth


def tiny_stream(seed, K, n, t_max):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.integers(0, t_max, n)).astype(np.uint32)
    ty = rng.integers(0, K, n).astype(np.uint8)
    return ty, t


def every_window(ty, t, K, widths):
    """max over every integer start x of the type-a events in [x, x + h]"""
    cap = np.zeros((K, len(widths)), np.uint32)
    for j, h in enumerate(widths):
        for x in range(int(t.min()) - int(h) - 1, int(t.max()) + 2):
            inside = (t.astype(np.int64) >= x) & (t.astype(np.int64) <= x + int(h))
            c = np.bincount(ty[inside], minlength=K)
            cap[:, j] = np.maximum(cap[:, j], c)
    return cap


@pytest.mark.parametrize("seed", range(6))
def test_capacity_equals_every_window_scan(seed):
    K = 3 + seed % 3
    ty, t = tiny_stream(seed, K, 40 + 7 * seed, 120)
    widths = [0, 1, 3, 7, 20, 55, 200]
    got = oracle.capacity_table(ty, t, K, widths)
    assert np.array_equal(got, every_window(ty, t, K, widths))


def test_capacity_closed_forms():
    ty, t = tiny_stream(99, 4, 300, 500)
    K = 5  # type 4 never occurs
    span = int(t.max() - t.min())
    cap = oracle.capacity_table(ty, t, K, [0, span, span + 1000, 1, 2, 40])
    hist = np.bincount(ty, minlength=K)
    # h = 0: the most events of one type at one time
    same = np.zeros(K, np.uint32)
    for a in range(K):
        _, c = np.unique(t[ty == a], return_counts=True)
        same[a] = c.max() if len(c) else 0
    assert np.array_equal(cap[:, 0], same)
    # a window as long as the stream holds every event of the type
    assert np.array_equal(cap[:, 1], hist) and np.array_equal(cap[:, 2], hist)
    assert cap[4].sum() == 0
    # monotone in the width
    order = np.argsort([0, span, span + 1000, 1, 2, 40], kind="stable")
    assert np.all(np.diff(cap[:, order].astype(np.int64), axis=1) >= 0)


@pytest.mark.parametrize("seed", range(4))
def test_capacity_bounds_mapconcat_entry_classes(seed):
    """Every exact MapConcatenate table (one segment per event, so every look-back
    window is tabulated) has at most 1 + cap[E_N, W] entries, and the largest window of
    last-node events that ends just before an event reaches the bound's count."""
    rng = np.random.default_rng(seed)
    K = 3
    ty, t = tiny_stream(50 + seed, K, 90, 400)
    N = 2 + seed % 3
    E = [int(x) for x in rng.choice(K, N, replace=seed % 2 == 0)]
    lo = [int(x) for x in rng.integers(0, 5, N - 1)]
    hi = [lo[k] + int(rng.integers(3, 30)) for k in range(N - 1)]
    W = int(sum(hi))
    bounds = np.arange(len(t) + 1)
    _, sizes = oracle.count_mapconcat(ty, t, E, lo, hi, bounds, return_sizes=True)
    cap = oracle.capacity_table(ty, t, K, [W])
    assert sizes.max() <= 1 + int(cap[E[-1], 0])
    # the table of segment L holds the last-node events with t[L] - W <= t < t[L]
    want = [1 + int(np.sum((ty[:L] == E[-1]) & (t[:L].astype(np.int64) >= int(t[L]) - W)))
            for L in range(len(t))]
    assert np.array_equal(sizes, want)


def test_capacity_on_a_bursting_recording():
    """Bursts at 200 Hz: a type holds several events in 20 ms there, against one or two
    in the 5 Hz background; the table sees the bursts."""
    cfg = synth.bursty_recording()
    s = cfg["stream"]
    cap = oracle.capacity_table(s.types, s.t, s.n_types, [20_000, 40_000, 1_000_000])
    assert cap[:, 0].min() >= 3
    assert np.all(cap[:, 1] >= cap[:, 0]) and np.all(cap[:, 2] >= cap[:, 1])
