"""A resident stream grown by fem_append_stream (Def. 2.1; a live recording delivered in
chunks, Section 1) counts and mines exactly like the whole stream loaded at once, and
the context's memory budget is enforced."""
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


def grown_stream(ctx, ty, t, K, cuts, device_every=2):
    """Load ty[:cuts[0]], then append the pieces between the cuts (some from device
    memory)."""
    torch = pytest.importorskip("torch")
    sid = fem.fem_load_stream(ctx, ty[:cuts[0]], t[:cuts[0]], K)
    bounds = list(cuts) + [len(t)]
    for k, (a, b) in enumerate(zip(bounds[:-1], bounds[1:])):
        if k % device_every == 1:
            fem.fem_append_stream(ctx, sid, torch.from_numpy(ty[a:b].copy()).cuda(),
                                  torch.from_numpy(t[a:b].view(np.int32).copy()).cuda())
        else:
            fem.fem_append_stream(ctx, sid, ty[a:b], t[a:b])
    return sid


def test_appended_stream_counts_equal_oracle(ctx):
    ty, t, K, _ = mid_stream()
    # pieces ending inside a chunk, exactly at a chunk end, one event, and many chunks
    cuts = [0, 1000, 2048, 2049, 4096, 4097, 9000, 30000]
    sid = grown_stream(ctx, ty, t, K, cuts)
    assert_counts_equal(fem.fem_type_counts(ctx, sid, K), np.bincount(ty, minlength=K),
                        "type counts")
    L, E, iv = synth.random_candidates(0xA1, 600, K, [2, 3, 4], 4)
    rec = fem.pack_episodes(L, E, iv)
    for p in (fem.PASS_RELAXED, fem.PASS_EXACT):
        want = oracle.count_batch(ty, t, L, E, iv, I_MS4,
                                  oracle.RELAXED if p == fem.PASS_RELAXED else oracle.EXACT)
        for seg in (0, 7):
            fem.fem_set_config(ctx, segments=seg)
            assert_counts_equal(fem.fem_count_candidates(ctx, sid, rec, I_MS4, p), want,
                                f"pass {p} segments {seg}")
    fem.fem_set_config(ctx, reset=True)
    got = fem.fem_mine_levelwise(ctx, sid, I_MS4, 60, 4)
    assert got == oracle.mine(ty, t, K, I_MS4, 60, 4)
    fem.fem_free_stream(ctx, sid)


def test_append_grows_past_capacity_and_rejects_bad_events(ctx):
    ty, t, K, _ = mid_stream(seed=0xFE12, T=20.0)
    sid = fem.fem_load_stream(ctx, ty[:100], t[:100], K)
    for a in range(100, len(t), 3000):  # many growths of the buffers
        fem.fem_append_stream(ctx, sid, ty[a:a + 3000], t[a:a + 3000])
    L, E, iv = synth.random_candidates(0xA2, 300, K, [2, 3], 4)
    rec = fem.pack_episodes(L, E, iv)
    want = oracle.count_batch(ty, t, L, E, iv, I_MS4, oracle.EXACT)
    assert_counts_equal(fem.fem_count_candidates(ctx, sid, rec, I_MS4, fem.PASS_EXACT), want,
                        "grown")
    # a time before the stream's last one, and a type out of range: nothing is appended
    with pytest.raises(fem.FemError) as e:
        fem.fem_append_stream(ctx, sid, np.array([1], np.uint8), np.array([t[-1] - 1], np.uint32))
    assert e.value.status == -2
    with pytest.raises(fem.FemError) as e:
        fem.fem_append_stream(ctx, sid, np.array([1, K], np.uint8),
                              np.array([t[-1], t[-1] + 5], np.uint32))
    assert e.value.status == -3
    assert_counts_equal(fem.fem_type_counts(ctx, sid, K), np.bincount(ty, minlength=K),
                        "histogram after rejected appends")
    assert_counts_equal(fem.fem_count_candidates(ctx, sid, rec, I_MS4, fem.PASS_EXACT), want,
                        "after rejected appends")
    with pytest.raises(fem.FemError) as e:
        fem.fem_append_stream(ctx, 12345, ty[:1], t[:1])
    assert e.value.status == -10
    fem.fem_free_stream(ctx, sid)


def test_memory_budget():
    ty, t, K, _ = mid_stream()
    budget = 320 << 10
    c = fem.fem_create(0, mem_budget_bytes=budget)
    try:
        small = 5000
        sid = fem.fem_load_stream(c, ty[:small], t[:small], K)
        used, b = fem.fem_mem_usage(c)
        assert b == budget and 0 < used <= budget
        with pytest.raises(fem.FemError) as e:  # ~40k events need about 530 KB
            fem.fem_load_stream(c, ty, t, K)
        assert e.value.status == -5
        assert fem.fem_mem_usage(c)[0] <= budget
        # the context stays usable within its budget
        L, E, iv = synth.random_candidates(0xA3, 200, K, [2, 3], 4)
        got = fem.fem_count_candidates(c, sid, fem.pack_episodes(L, E, iv), I_MS4, fem.PASS_EXACT)
        assert_counts_equal(got, oracle.count_batch(ty[:small], t[:small], L, E, iv, I_MS4,
                                                    oracle.EXACT), "within budget")
        fem.fem_free_stream(c, sid)
    finally:
        fem.fem_destroy(c)
