"""The capacity table computed on the GPU (fem_capacity_table) equals the oracle's,
element by element: the most events of each type in one closed window of each width,
the bound on Algorithm 1's lists (Section 5.1) and on the MapConcatenate entry classes
(Section 5.2.2)."""
import numpy as np
import pytest

import oracle
from paper_0905_2200_gb300 import fem, synth
from tests.gpu_common import assert_counts_equal, ctx_fixture, mid_stream

pytestmark = pytest.mark.gpu

WIDTHS = [0, 1, 2_000, 5_000, 20_000, 40_000, 140_000, 1_000_000, 0xFFFFFFFF]


@pytest.fixture(scope="module")
def ctx():
    c = ctx_fixture()
    yield c
    fem.fem_destroy(c)


def check(ctx, ty, t, K, widths=WIDTHS, what=""):
    sid = fem.fem_load_stream(ctx, ty, t, K)
    try:
        got = fem.fem_capacity_table(ctx, sid, widths, K)
        want = oracle.capacity_table(ty, t, K, widths)
        assert_counts_equal(got.reshape(-1), want.reshape(-1), what)
    finally:
        fem.fem_free_stream(ctx, sid)


def test_capacity_mid_stream(ctx):
    ty, t, K, _ = mid_stream()
    check(ctx, ty, t, K, what="mid stream")


def test_capacity_equal_times_absent_types_and_one_chunk(ctx):
    rng = np.random.default_rng(7)
    n = 1500  # less than one chunk
    t = np.sort(rng.integers(0, 3_000, n)).astype(np.uint32)  # many equal times
    ty = rng.integers(0, 5, n).astype(np.uint8)  # types 5..9 never occur
    check(ctx, ty, t, 10, widths=[0, 1, 2, 7, 100, 2_999, 3_000], what="equal times")


def test_capacity_bursting_recording(ctx):
    cfg = synth.bursty_recording()
    s = cfg["stream"]
    check(ctx, s.types, s.t, s.n_types, what="bursts")


def test_capacity_benchmark_recording(ctx):
    cfg = synth.single_recording()
    s = cfg["stream"]
    hi = sorted({int(h) for _, h in cfg["intervals"]})
    widths = hi + [sum(hi[-1:]) * k for k in range(2, 8)]  # each hi and (N - 1) x the largest
    check(ctx, s.types, s.t, s.n_types, widths=widths, what="64-type recording")


def test_capacity_grown_stream_and_errors(ctx):
    ty, t, K, _ = mid_stream(seed=0xCA7, T=20.0)
    sid = fem.fem_load_stream(ctx, ty[:5000], t[:5000], K)
    fem.fem_append_stream(ctx, sid, ty[5000:], t[5000:])
    got = fem.fem_capacity_table(ctx, sid, WIDTHS, K)
    assert_counts_equal(got.reshape(-1), oracle.capacity_table(ty, t, K, WIDTHS).reshape(-1),
                        "grown")
    with pytest.raises(fem.FemError) as e:
        fem.fem_capacity_table(ctx, sid, [], K)
    assert e.value.status == -1
    with pytest.raises(fem.FemError) as e:
        fem.fem_capacity_table(ctx, sid, list(range(65)), K)
    assert e.value.status == -1
    fem.fem_free_stream(ctx, sid)
    with pytest.raises(fem.FemError) as e:
        fem.fem_capacity_table(ctx, sid, WIDTHS, K)
    assert e.value.status == -10
