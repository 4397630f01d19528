"""MapConcatenate as Section 5.2.2 prints it, on the device, against the oracle's
version of the same scheme (bit-exact, same time cuts), and its divergence from the
exact counts measured on the same inputs."""
import numpy as np
import pytest

import oracle
from paper_0905_2200_gb300 import fem, synth
from tests.gpu_common import I_MS4, assert_counts_equal, ctx_fixture, mid_stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = ctx_fixture()
    yield c
    fem.fem_destroy(c)


def time_cuts(t, segments):
    """The library's rule: cut at the first event of every ceil(chunks / P)-th chunk."""
    n = len(t)
    n_chunks = (n + 2047) // 2048
    P0 = max(1, min(segments, n_chunks))
    cps = (n_chunks + P0 - 1) // P0
    tau = [int(t[0]) - 1]
    for c0 in range(cps, n_chunks, cps):
        x = int(t[c0 * 2048]) - 1
        if tau[-1] < x < int(t[-1]):
            tau.append(x)
    tau.append(int(t[-1]))
    return tau


def oracle_literal(ty, t, L, E, iv, I, tau):
    lo, hi = oracle.resolve(L, E, iv, I)
    out, diag = [], [0, 0]
    for i in range(len(L)):
        N = int(L[i])
        c, _, d = oracle.count_mapconcat_literal(ty, t, E[i, :N], lo[i, :N - 1], hi[i, :N - 1], tau)
        out.append(c)
        diag[0] += d[0]
        diag[1] += d[1]
    return np.array(out, np.uint32), tuple(diag)


@pytest.mark.parametrize("segments", [1, 2, 7, 19])
def test_printed_mapconcat_equals_oracle(ctx, segments):
    ty, t, K, _ = mid_stream()
    sid = fem.fem_load_stream(ctx, ty, t, K)
    L, E, iv = synth.random_candidates(0x11 + segments, 300, K, [1, 2, 3, 4, 5], 4)
    got, diag = fem.fem_count_mapconcat_literal(ctx, sid, fem.pack_episodes(L, E, iv), I_MS4,
                                                segments)
    want, wdiag = oracle_literal(ty, t, L, E, iv, I_MS4, time_cuts(t, segments))
    assert_counts_equal(got, want, f"printed scheme P={segments}")
    assert diag == wdiag
    exact = fem.fem_count_candidates(ctx, sid, fem.pack_episodes(L, E, iv), I_MS4, fem.PASS_EXACT)
    assert np.all(got <= exact)            # it never counted more here
    if segments == 1:
        assert_counts_equal(got, exact, "one segment is Algorithm 1")
    fem.fem_free_stream(ctx, sid)


def test_printed_mapconcat_dense_stream_diverges_like_the_oracle(ctx):
    """A dense stream (gaps of 0-2 us, intervals of a few us) cut into three segments:
    boundaries with no or several matching tuples occur, the printed scheme loses an
    occurrence for one candidate, and the device reproduces the oracle exactly."""
    ty, t = synth.tiny_stream(77, 6000, 3, 2, tie_prob=0.3)
    sid = fem.fem_load_stream(ctx, ty, t, 3)
    I = np.array([[0, 3], [1, 6], [2, 8]], np.uint32)
    L, E, iv = synth.random_candidates(5, 200, 3, [2, 3], 3)
    exact = fem.fem_count_candidates(ctx, sid, fem.pack_episodes(L, E, iv), I, fem.PASS_EXACT)
    got, diag = fem.fem_count_mapconcat_literal(ctx, sid, fem.pack_episodes(L, E, iv), I, 3)
    want, wdiag = oracle_literal(ty, t, L, E, iv, I, time_cuts(t, 3))
    assert_counts_equal(got, want, "dense short stream")
    assert diag == wdiag and diag[0] > 0 and diag[1] > 0
    assert np.all(got <= exact) and np.any(got < exact)
    fem.fem_free_stream(ctx, sid)


def test_printed_mapconcat_rejects_repeated_types(ctx):
    ty, t, K, _ = mid_stream()
    sid = fem.fem_load_stream(ctx, ty, t, K)
    L, E, iv = synth.random_candidates(3, 20, 4, [3], 4, distinct=False)
    E[:, 1] = E[:, 0]
    with pytest.raises(fem.FemError) as e:
        fem.fem_count_mapconcat_literal(ctx, sid, fem.pack_episodes(L, E, iv), I_MS4, 4)
    assert e.value.status == -1
    fem.fem_free_stream(ctx, sid)
