"""Window-based frequency (Section 2's alternative measure) on the device against the
oracle's recurrence (itself pinned by brute force)."""
import numpy as np
import pytest

import oracle
from paper_0905_2200_gb300 import fem, synth
from tests.gpu_common import I_MS4, ctx_fixture, mid_stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = ctx_fixture()
    yield c
    fem.fem_destroy(c)


@pytest.mark.parametrize("w_us", [1, 4_000, 30_000, 250_000])
def test_window_counts_equal_oracle(ctx, w_us):
    ty, t, K, _ = mid_stream()
    sid = fem.fem_load_stream(ctx, ty, t, K)
    L, E, iv = synth.random_candidates(0x51, 240, K, [1, 2, 3, 4, 5], 4)
    got = fem.fem_count_windows(ctx, sid, fem.pack_episodes(L, E, iv), I_MS4, w_us)
    want = oracle.count_windows_batch(ty, t, L, E, iv, I_MS4, w_us)
    assert np.array_equal(got, want)
    assert (got > 0).any()
    fem.fem_free_stream(ctx, sid)


def test_window_counts_full_recording_sampled(ctx):
    """All 16,128 level-2 candidates of the 64-type recording with 40 ms windows; 64
    sampled candidates re-derived by the oracle; a longer window never covers fewer
    starts."""
    cfg = synth.single_recording()
    s = cfg["stream"]
    sid = fem.fem_load_stream(ctx, s.types, s.t, s.n_types)
    L, E, iv = synth.level2_candidates(range(64), 4)
    rec = fem.pack_episodes(L, E, iv)
    got = fem.fem_count_windows(ctx, sid, rec, cfg["intervals"], 40_000)
    wider = fem.fem_count_windows(ctx, sid, rec, cfg["intervals"], 80_000)
    assert np.all(wider >= got)
    pick = np.random.default_rng(4).choice(len(L), 64, replace=False)
    want = oracle.count_windows_batch(s.types, s.t, L[pick], E[pick], iv[pick], cfg["intervals"],
                                      40_000)
    assert np.array_equal(got[pick], want)
    fem.fem_free_stream(ctx, sid)
