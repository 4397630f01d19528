"""Parity of the CUDA counting kernels with the CPU oracle, element by element.

Covers both passes, every episode length 1..8, single-segment and segmented
(MapConcatenate) launches, the capacity-retry path, device buffers, edge cases
and error statuses.  Inputs are seeded synthetic streams (see synth.py).
"""
import numpy as np
import pytest

import oracle
from paper_0905_2200_gb300 import fem, synth
from tests.gpu_common import I_MS4, assert_counts_equal, ctx_fixture, mid_stream, oracle_counts

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
def tiny(ctx):
    cfg = synth.tiny_mining()
    s = cfg["stream"]
    sid = fem.fem_load_stream(ctx, s.types, s.t, s.n_types)
    return s, sid


@pytest.fixture(scope="module")
def mid(ctx):
    ty, t, K, chains = mid_stream()
    sid = fem.fem_load_stream(ctx, ty, t, K)
    return ty, t, K, chains, sid


def test_type_counts_match_histogram(ctx, tiny):
    s, sid = tiny
    assert np.array_equal(fem.fem_type_counts(ctx, sid, s.n_types),
                          np.bincount(s.types, minlength=s.n_types))


@pytest.mark.parametrize("pass_", PASSES)
def test_every_length_tiny(ctx, tiny, pass_):
    s, sid = tiny
    I = np.array([[4000, 6000], [0, 3000], [1000, 9000]], np.uint32)
    L, E, iv = synth.random_candidates(31, 1600, s.n_types, [1, 2, 3, 4, 5, 6, 7, 8], len(I))
    got = fem.fem_count_candidates(ctx, sid, fem.pack_episodes(L, E, iv), I, pass_)
    assert_counts_equal(got, oracle_counts(s.types, s.t, L, E, iv, I, pass_), "tiny")


@pytest.mark.parametrize("pass_", PASSES)
@pytest.mark.parametrize("segments", [1, 2, 3, 7, 19])
def test_segmented_equals_oracle(ctx, mid, pass_, segments):
    ty, t, K, chains, sid = mid
    L, E, iv = synth.random_candidates(77 + segments, 700, K, [2, 3, 4, 5, 6], 4)
    rec = fem.pack_episodes(L, E, iv)
    fem.fem_set_config(ctx, segments=segments)
    got = fem.fem_count_candidates(ctx, sid, rec, I_MS4, pass_)
    assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I_MS4, pass_), f"P={segments}")


@pytest.mark.parametrize("pass_", PASSES)
@pytest.mark.parametrize("segments", [1, 5])
def test_mixed_interval_widths(ctx, mid, pass_, segments):
    """Edges with hi >= 2 lo (two live clusters per list at most: register lists) next
    to edges with hi < 2 lo (more live clusters: shared-memory rings), in one warp."""
    ty, t, K, chains, sid = mid
    I = np.array([[0, 2000], [4000, 6000], [2000, 5000], [9000, 11000], [5000, 10000]],
                 np.uint32)
    L, E, iv = synth.random_candidates(0x31 + segments, 900, K, [2, 3, 4, 5], len(I))
    fem.fem_set_config(ctx, segments=segments)
    got = fem.fem_count_candidates(ctx, sid, fem.pack_episodes(L, E, iv), I, pass_)
    assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I, pass_), f"mixed P={segments}")


@pytest.mark.parametrize("pass_", PASSES)
def test_autotuned_launch_level2_mid(ctx, mid, pass_):
    ty, t, K, chains, sid = mid
    L, E, iv = synth.level2_candidates(range(K), 4)
    got = fem.fem_count_candidates(ctx, sid, fem.pack_episodes(L, E, iv), I_MS4, pass_)
    assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I_MS4, pass_), "level2 mid")


@pytest.mark.parametrize("pass_", PASSES)
def test_dense_completions_wide_windows(ctx, pass_):
    """Few types at a high rate with second-long intervals: completions are dense, the
    look-back window spans several chunks and holds more entry classes than a table
    has slots, so the recount path runs too."""
    t, ty = synth.poisson_stream(0xD0, 3, 200.0, 40.0)
    sid = fem.fem_load_stream(ctx, ty, t, 3)
    I = np.array([[0, 2_000_000], [50_000, 900_000], [0, 30_000]], np.uint32)
    L, E, iv = synth.random_candidates(5, 120, 3, [1, 2, 3], 3)
    rec = fem.pack_episodes(L, E, iv)
    want = oracle_counts(ty, t, L, E, iv, I, pass_)
    for P in (1, 4, 11):
        fem.fem_set_config(ctx, segments=P)
        got = fem.fem_count_candidates(ctx, sid, rec, I, pass_)
        assert_counts_equal(got, want, f"dense P={P}")
    fem.fem_free_stream(ctx, sid)


def test_exact_ring_overflow_is_recounted(ctx):
    """Bursts of 300 events of one type inside one interval: rings of 16/32 overflow and
    the library recounts with a larger ring (or reports FEM_EOVERFLOW, never a wrong count)."""
    ty, t = [], []
    cur = 0
    for b in range(20):
        cur += 1_000_000
        for j in range(100):
            ty.append(0)
            t.append(cur + j * 10)
        ty.append(1)
        t.append(cur + 5_000)
    ty, t = np.array(ty, np.uint8), np.array(t, np.uint32)
    sid = fem.fem_load_stream(ctx, ty, t, 2)
    I = np.array([[4_000, 6_000], [0, 10_000]], np.uint32)
    L = np.array([2, 2], np.uint8)
    E = np.zeros((2, 8), np.uint8)
    E[:, 1] = 1
    iv = np.zeros((2, 7), np.uint8)
    iv[1, 0] = 1
    got = fem.fem_count_candidates(ctx, sid, fem.pack_episodes(L, E, iv), I, fem.PASS_EXACT)
    assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I, fem.PASS_EXACT), "burst")
    fem.fem_free_stream(ctx, sid)


@pytest.mark.parametrize("threads", [256, 32])
def test_recount_block_size_fits_its_rings(ctx, threads):
    """Overflowing episodes are recounted with larger rings; the recount picks a block
    size its shared memory can hold, whatever size is configured for the first count
    (here with three segments, so the segmented recount runs)."""
    ty, t = [], []
    cur = 0
    for b in range(12):              # 12 bursts of 600 events: four chunks, cut in bursts
        cur += 1_000_000
        for j in range(600):
            ty.append(j % 3)
            t.append(cur + j * 10)
        ty.append(3)
        t.append(cur + 5_000)
    order = np.argsort(np.array(t), kind="stable")
    ty, t = np.array(ty, np.uint8)[order], np.array(t, np.uint32)[order]
    sid = fem.fem_load_stream(ctx, ty, t, 4)
    I = np.array([[4_000, 6_000], [0, 10_000], [1_000, 9_000]], np.uint32)
    L, E, iv = synth.random_candidates(71, 60, 4, [2, 3, 4], 3)
    fem.fem_set_config(ctx, segments=3, threads_per_block=threads)
    got = fem.fem_count_candidates(ctx, sid, fem.pack_episodes(L, E, iv), I, fem.PASS_EXACT)
    fem.fem_set_config(ctx, reset=True)
    assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I, fem.PASS_EXACT), f"T={threads}")
    fem.fem_free_stream(ctx, sid)


@pytest.mark.parametrize("pass_", PASSES)
def test_repeated_types_use_single_segment_path(ctx, mid, pass_):
    ty, t, K, chains, sid = mid
    L, E, iv = synth.random_candidates(9, 300, 4, [2, 3, 4], 4, distinct=False)
    got = fem.fem_count_candidates(ctx, sid, fem.pack_episodes(L, E, iv), I_MS4, pass_)
    assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I_MS4, pass_), "repeats")


def test_two_pass_matches_algorithm_4(ctx, mid):
    ty, t, K, chains, sid = mid
    L, E, iv = synth.level2_candidates(range(K), 4)
    theta = 60
    ex, sv = fem.fem_count_two_pass(ctx, sid, fem.pack_episodes(L, E, iv), I_MS4, theta)
    rel_o, ex_o, sv_o = oracle.two_pass(ty, t, L, E, iv, I_MS4, theta)
    assert_counts_equal(sv, sv_o, "survived")
    assert_counts_equal(ex, ex_o, "exact")
    assert 0 < sv.sum() < len(sv)


def test_device_tensors_in_and_out(ctx, mid):
    torch = pytest.importorskip("torch")
    ty, t, K, chains, sid = mid
    sid2 = fem.fem_load_stream(ctx, torch.from_numpy(ty).cuda(), torch.from_numpy(t).cuda(), K)
    L, E, iv = synth.random_candidates(3, 900, K, [2, 3, 4], 4)
    rec = torch.from_numpy(fem.pack_episodes(L, E, iv)).cuda()
    out = torch.zeros(900, dtype=torch.int32, device="cuda")
    fem.fem_count_candidates(ctx, sid2, rec, I_MS4, fem.PASS_EXACT, out=out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I_MS4, fem.PASS_EXACT), "device")
    fem.fem_free_stream(ctx, sid2)


def test_device_load_checks_and_copies(ctx):
    """A stream loaded from device memory is checked, copied and grouped by one kernel:
    an inversion across a chunk's end and a type >= K are rejected, and a valid stream
    has the type counts and episode counts of the same stream loaded from host memory."""
    torch = pytest.importorskip("torch")
    K = 5
    ty, t = synth.tiny_stream(7, 5000, K, 300, tie_prob=0.2)
    assert t[2047] > 0
    t_bad = t.copy()
    t_bad[2048] = t_bad[2047] - 1  # the pair across the first chunk's end
    ty_bad = ty.copy()
    ty_bad[4999] = K  # the last event of the ragged last chunk
    for tt, yy, status in ((t_bad, ty, -2), (t, ty_bad, -3)):
        with pytest.raises(fem.FemError) as e:
            fem.fem_load_stream(ctx, torch.from_numpy(yy).cuda(), torch.from_numpy(tt).cuda(), K)
        assert e.value.status == status
    sid_d = fem.fem_load_stream(ctx, torch.from_numpy(ty).cuda(), torch.from_numpy(t).cuda(), K)
    sid_h = fem.fem_load_stream(ctx, ty, t, K)
    assert np.array_equal(fem.fem_type_counts(ctx, sid_d, K), np.bincount(ty, minlength=K))
    L, E, iv = synth.random_candidates(4, 300, K, [1, 2, 3], 2)
    rec = fem.pack_episodes(L, E, iv)
    I = np.array([[0, 400], [200, 900]], np.uint32)
    for p in PASSES:
        got_d = fem.fem_count_candidates(ctx, sid_d, rec, I, p)
        got_h = fem.fem_count_candidates(ctx, sid_h, rec, I, p)
        assert np.array_equal(got_d, got_h)
        assert_counts_equal(got_d, oracle_counts(ty, t, L, E, iv, I, p), "device load")
    fem.fem_free_stream(ctx, sid_d)
    fem.fem_free_stream(ctx, sid_h)


# ------------------------------------------------------------------------ edge cases
def test_empty_and_tiny_streams(ctx):
    I = np.array([[0, 1000]], np.uint32)
    L, E, iv = synth.random_candidates(1, 50, 3, [1, 2, 3], 1)
    rec = fem.pack_episodes(L, E, iv)
    for n in (0, 1, 2, 5, 2047, 2048, 2049):
        ty, t = synth.tiny_stream(n + 3, n, 3, 300, tie_prob=0.3)
        sid = fem.fem_load_stream(ctx, ty, t, 3)
        for p in PASSES:
            got = fem.fem_count_candidates(ctx, sid, rec, I, p)
            assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I, p), f"n={n}")
        fem.fem_free_stream(ctx, sid)


def test_all_equal_times(ctx):
    ty = np.array([0, 1, 2] * 700, np.uint8)
    t = np.full(ty.shape, 12345, np.uint32)
    sid = fem.fem_load_stream(ctx, ty, t, 3)
    I = np.array([[0, 5]], np.uint32)
    L, E, iv = synth.random_candidates(2, 40, 3, [1, 2, 3], 1)
    for p in PASSES:
        got = fem.fem_count_candidates(ctx, sid, fem.pack_episodes(L, E, iv), I, p)
        assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I, p), "ties")
    fem.fem_free_stream(ctx, sid)


def test_zero_candidates(ctx, tiny):
    s, sid = tiny
    out = fem.fem_count_candidates(ctx, sid, np.zeros((0, 16), np.uint8), [[0, 5]])
    assert out.shape == (0,)


def test_error_statuses(ctx, tiny):
    s, sid = tiny
    with pytest.raises(fem.FemError) as e:
        fem.fem_load_stream(ctx, np.array([0, 1], np.uint8), np.array([5, 4], np.uint32), 2)
    assert e.value.status == -2
    with pytest.raises(fem.FemError) as e:
        fem.fem_load_stream(ctx, np.array([0, 7], np.uint8), np.array([4, 5], np.uint32), 4)
    assert e.value.status == -3
    rec = fem.pack_episodes([2], [[0, 1, 0, 0, 0, 0, 0, 0]], [[0] * 7])
    for bad_I in ([[5, 5]], [[6, 5]]):
        with pytest.raises(fem.FemError) as e:
            fem.fem_count_candidates(ctx, sid, rec, bad_I)
        assert e.value.status == -1
    for bad in (fem.pack_episodes([0], [[0] * 8], [[0] * 7]),
                fem.pack_episodes([9], [[0] * 8], [[0] * 7]),
                fem.pack_episodes([2], [[0, 99, 0, 0, 0, 0, 0, 0]], [[0] * 7]),
                fem.pack_episodes([2], [[0, 1, 0, 0, 0, 0, 0, 0]], [[3, 0, 0, 0, 0, 0, 0]])):
        with pytest.raises(fem.FemError) as e:
            fem.fem_count_candidates(ctx, sid, bad, [[0, 5]])
        assert e.value.status == -1
    with pytest.raises(fem.FemError) as e:
        fem.fem_count_candidates(ctx, sid, rec, [[0, 0xFFFFFFF0]])
    assert e.value.status == -4
    with pytest.raises(fem.FemError) as e:
        fem.fem_count_candidates(ctx, 999, rec, [[0, 5]])
    assert e.value.status == -10
