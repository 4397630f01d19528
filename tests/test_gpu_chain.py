"""The latest-chain counting kernels (prefix lists shared by a block's candidates) against
the oracle, element by element, next to the per-thread machine kernels: both passes,
lengths 2..8, one segment and MapConcatenate segments, the fallbacks (more prefixes
than a block's node table, lists longer than a chunk's capacity, exact look-ups past a
full carried tail) and level-wise mining.  Algorithms 1 and 3 (Sections 5.1, 5.3.1);
MapConcatenate (Section 5.2.2)."""
import numpy as np
import pytest

import oracle
from paper_0905_2200_gb300 import fem, synth
from tests.gpu_common import (I_MS4, assert_counts_equal, ctx_fixture, mid_stream,
                              mining_stream, oracle_counts)

pytestmark = pytest.mark.gpu
PASSES = (fem.PASS_RELAXED, fem.PASS_EXACT)


@pytest.fixture(scope="module")
def ctx():
    c = ctx_fixture()
    yield c
    fem.fem_destroy(c)


@pytest.fixture(autouse=True)
def _reset_config(ctx):
    fem.fem_set_config(ctx, reset=True)
    yield
    fem.fem_set_config(ctx, reset=True)


@pytest.fixture(scope="module")
def mid(ctx):
    ty, t, K, chains = mid_stream()
    sid = fem.fem_load_stream(ctx, ty, t, K)
    return ty, t, K, sid


def families(seed, K, N, n_prefix, children, n_int=4):
    """Candidates in canonical order that share prefixes: n_prefix random (N-1)-node
    prefixes, each extended by up to `children` random (interval, new type) pairs."""
    rng = np.random.default_rng(seed)
    rows = set()
    for _ in range(n_prefix):
        pre = [int(x) for x in rng.choice(K, N - 1, replace=False)]
        piv = [int(x) for x in rng.integers(0, n_int, N - 2)]
        rest = [x for x in range(K) if x not in pre]
        for _ in range(int(rng.integers(1, children + 1))):
            b = int(rng.choice(rest))
            key = []
            ivs = piv + [int(rng.integers(0, n_int))]
            for k in range(N):
                key.append((pre + [b])[k])
                if k < N - 1:
                    key.append(ivs[k])
            rows.add(tuple(key))
    rows = sorted(rows)
    m = len(rows)
    L = np.full(m, N, np.uint8)
    E = np.zeros((m, 8), np.uint8)
    iv = np.zeros((m, 7), np.uint8)
    for i, r in enumerate(rows):
        E[i, :N] = r[0::2]
        iv[i, :N - 1] = r[1::2]
    return L, E, iv


@pytest.mark.parametrize("pass_", PASSES)
@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("segments", [1, 3, 19])
def test_chain_equals_oracle(ctx, mid, pass_, N, segments):
    ty, t, K, sid = mid
    L, E, iv = families(1000 * N + segments, K, N, 60, 12)
    rec = fem.pack_episodes(L, E, iv)
    want = oracle_counts(ty, t, L, E, iv, I_MS4, pass_)
    for kernel in (fem.KERNEL_CHAIN, fem.KERNEL_MACHINE):
        fem.fem_set_config(ctx, segments=segments, kernel=kernel)
        got = fem.fem_count_candidates(ctx, sid, rec, I_MS4, pass_)
        assert_counts_equal(got, want, f"kernel {kernel} N={N} P={segments}")


@pytest.mark.parametrize("pass_", PASSES)
@pytest.mark.parametrize("threads", [32, 64, 128, 256])
def test_chain_block_sizes_and_ragged_tail(ctx, mid, pass_, threads):
    """Block sizes 32..256 over a candidate count that leaves a ragged last block."""
    ty, t, K, sid = mid
    L, E, iv = families(77 + threads, K, 3, 97, 9)
    rec = fem.pack_episodes(L, E, iv)
    fem.fem_set_config(ctx, threads_per_block=threads, kernel=fem.KERNEL_CHAIN, segments=5)
    got = fem.fem_count_candidates(ctx, sid, rec, I_MS4, pass_)
    assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I_MS4, pass_), f"T={threads}")


@pytest.mark.parametrize("pass_", PASSES)
@pytest.mark.parametrize("N", [2, 3, 4])
@pytest.mark.parametrize("segments", [1, 6])
def test_chain_many_prefixes_counted_in_parts(ctx, mid, pass_, N, segments):
    """A block whose candidates have more distinct prefixes than its node tables hold
    counts them in parts (runs of prefixes, the segment streamed once per part)."""
    ty, t, K, sid = mid
    L, E, iv = families(0x5A + 10 * N + segments, K, N, 300, 1 if N > 2 else 3)
    rec = fem.pack_episodes(L, E, iv)
    fem.fem_set_config(ctx, kernel=fem.KERNEL_CHAIN, segments=segments)
    got = fem.fem_count_candidates(ctx, sid, rec, I_MS4, pass_)
    assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I_MS4, pass_), f"parts N={N}")


@pytest.mark.parametrize("pass_", PASSES)
def test_chain_unshared_prefixes_fall_back(ctx, mid, pass_):
    """Random (unsorted) candidates: a block sees more distinct prefixes than its node
    table holds; those candidates are recounted by the per-thread kernels."""
    ty, t, K, sid = mid
    L, E, iv = synth.random_candidates(0xC4, 900, K, [2, 3, 4], 4)
    fem.fem_set_config(ctx, kernel=fem.KERNEL_CHAIN, segments=4)
    got = fem.fem_count_candidates(ctx, sid, fem.pack_episodes(L, E, iv), I_MS4, pass_)
    assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I_MS4, pass_), "unsorted")


@pytest.mark.parametrize("pass_", PASSES)
def test_chain_dense_lists_fall_back(ctx, pass_):
    """Three types at 300 Hz with wide intervals: a prefix admits more events per chunk
    than a list holds and exact look-ups walk past full carried tails (the fallback),
    with equal times among the events."""
    t, ty = synth.poisson_stream(0xD3, 3, 300.0, 20.0)
    t = (t // 50) * 50  # many equal times
    sid = fem.fem_load_stream(ctx, ty, t, 3)
    I = np.array([[0, 40_000], [20_000, 30_000], [0, 400]], np.uint32)
    L, E, iv = families(5, 3, 3, 6, 6, n_int=3)
    L2, E2, iv2 = families(6, 3, 2, 3, 6, n_int=3)
    rec = fem.pack_episodes(L, E, iv)
    rec2 = fem.pack_episodes(L2, E2, iv2)
    for P in (1, 6):
        fem.fem_set_config(ctx, kernel=fem.KERNEL_CHAIN, segments=P)
        got = fem.fem_count_candidates(ctx, sid, rec, I, pass_)
        assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I, pass_), f"dense N=3 P={P}")
        got2 = fem.fem_count_candidates(ctx, sid, rec2, I, pass_)
        assert_counts_equal(got2, oracle_counts(ty, t, L2, E2, iv2, I, pass_), f"dense N=2 P={P}")
    fem.fem_free_stream(ctx, sid)


@pytest.mark.parametrize("kernel", [fem.KERNEL_CHAIN, fem.KERNEL_MACHINE])
@pytest.mark.parametrize("segments", [0, 1, 4])
def test_mining_with_each_kernel(ctx, kernel, segments):
    ty, t, K, _ = mining_stream()
    sid = fem.fem_load_stream(ctx, ty, t, K)
    fem.fem_set_config(ctx, kernel=kernel, segments=segments)
    got = fem.fem_mine_levelwise(ctx, sid, I_MS4, 80, 6)
    assert got == oracle.mine(ty, t, K, I_MS4, 80, 6)
    fem.fem_free_stream(ctx, sid)
