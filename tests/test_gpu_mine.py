"""Parity of the on-device level-wise miner (candidate generation, two-pass counting,
compaction, join) with the oracle's miner, and sampled full-size checks."""
import numpy as np
import pytest

import oracle
from paper_0905_2200_gb300 import fem, synth
from tests.gpu_common import I_MS4, assert_counts_equal, ctx_fixture, mining_stream

pytestmark = pytest.mark.gpu


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


def test_mine_tiny_equals_oracle(ctx):
    cfg = synth.tiny_mining()
    s = cfg["stream"]
    sid = fem.fem_load_stream(ctx, s.types, s.t, s.n_types)
    got = fem.fem_mine_levelwise(ctx, sid, cfg["intervals"], cfg["theta"], cfg["max_len"])
    want = oracle.mine(s.types, s.t, s.n_types, cfg["intervals"], cfg["theta"], cfg["max_len"])
    assert got == want
    assert any(r[0] == (0, 1, 2, 3) for r in got[4])
    stats = fem.fem_last_mine_stats(ctx)
    assert stats[0]["level"] == 2 and stats[0]["candidates"] == 16 * 15


@pytest.mark.parametrize("theta,segments", [(150, 0), (80, 0), (80, 1), (80, 3), (150, 10)])
def test_mine_chains_equals_oracle(ctx, theta, segments):
    ty, t, K, chains = mining_stream()
    sid = fem.fem_load_stream(ctx, ty, t, K)
    if segments:
        fem.fem_set_config(ctx, segments=segments)
    got = fem.fem_mine_levelwise(ctx, sid, I_MS4, theta, 6)
    want = oracle.mine(ty, t, K, I_MS4, theta, 6)
    assert got == want
    assert max(got) == 6
    fem.fem_free_stream(ctx, sid)


def test_mine_edge_cases(ctx):
    I = np.array([[0, 1000]], np.uint32)
    # empty stream, a stream where nothing is frequent, max_len 1
    for n, theta, max_len in ((0, 1, 4), (50, 10**6, 4), (500, 5, 1), (500, 3, 2)):
        ty, t = synth.tiny_stream(n, n, 3, 300)
        sid = fem.fem_load_stream(ctx, ty, t, 3)
        got = fem.fem_mine_levelwise(ctx, sid, I, theta, max_len)
        want = oracle.mine(ty, t, 3, I, theta, max_len)
        assert got == {k: v for k, v in want.items() if v}
        fem.fem_free_stream(ctx, sid)


@pytest.mark.parametrize("segments", [0, 3])
def test_mine_repeated_types_equals_oracle(ctx, segments):
    """Mining with repeated types allowed, on a stream with the chains A -> B -> A and
    C -> D -> C -> E: the repeat-keeping miner equals the oracle's (candidate sets with
    both distinct and repeated types are split, the repeated ones counted with one
    segment)."""
    t, ty = synth.poisson_stream(0xAB, 10, 8.0, 30.0,
                                 chains=[((0, 1, 0), 3.0, [(2000, 5000), (5000, 10000)]),
                                         ((2, 3, 2, 4), 2.0, [(0, 2000), (2000, 5000),
                                                              (10000, 20000)])])
    sid = fem.fem_load_stream(ctx, ty, t, 10)
    if segments:
        fem.fem_set_config(ctx, segments=segments)
    got = fem.fem_mine_levelwise(ctx, sid, I_MS4, 40, 5, repeated_types=True)
    want = oracle.mine(ty, t, 10, I_MS4, 40, 5, repeated_types=True)
    assert got == want
    assert any(len(set(r[0])) < len(r[0]) for lv in got.values() for r in lv)
    assert max(got) >= 3
    fem.fem_free_stream(ctx, sid)


@pytest.mark.parametrize("theta", [1300, 4000])
@pytest.mark.parametrize("segments", [0, 40])
def test_mine_bursts_level2_pairs_equals_oracle(ctx, segments, theta):
    """Level 2's relaxed pass runs on the pair kernel (every interval variant of an
    ordered type pair in one thread).  In bursts hundreds of candidates need more entry
    classes than its four slots -- more than 1/64 of the level -- so they are recounted
    before the elimination: the mined sets and the level-2 survivors equal the oracle's
    (at theta 4000, above every relaxed count, there are none).  Stream: the bursting
    recording's types 0, 4, ..., 60 (96k events)."""
    cfg = synth.bursty_recording()
    s, I = cfg["stream"], cfg["intervals"]
    keep = (s.types % 4) == 0
    ty, t = (s.types[keep] // 4).astype(np.uint8), s.t[keep]
    sid = fem.fem_load_stream(ctx, ty, t, 16)
    fem.fem_set_config(ctx, segments=segments)
    got = fem.fem_mine_levelwise(ctx, sid, I, theta, 3)
    stats = fem.fem_last_mine_stats(ctx)
    fem.fem_free_stream(ctx, sid)
    want = oracle.mine(ty, t, 16, I, theta, 3)
    assert got == want
    L, E, iv = synth.level2_candidates(range(16), len(I))
    rel = oracle.count_batch(ty, t, L, E, iv, I, oracle.RELAXED)
    assert stats[0]["level"] == 2 and stats[0]["kernel_relaxed"] == fem.KERNEL_PAIRS
    assert stats[0]["survivors"] == int((rel >= theta).sum())


def test_mine_few_flagged_pass_to_exact(ctx):
    """A quiet 16-type stream with six 100 ms bursts, four segments: 15 level-2
    candidates (960 / 64) need more entry classes than the pair kernel's slots.  So few
    go to the exact pass unfiltered -- their relaxed counts are below theta, so the
    oracle eliminates them -- and the exact pass drops them again: the mined sets equal
    the oracle's and the level-2 survivors are the oracle's plus those 15."""
    ty, t = synth.sparse_bursts()
    I, theta = synth.I_BURST.copy(), 400
    sid = fem.fem_load_stream(ctx, ty, t, 16)
    fem.fem_set_config(ctx, segments=4)
    got = fem.fem_mine_levelwise(ctx, sid, I, theta, 3)
    stats = fem.fem_last_mine_stats(ctx)
    fem.fem_free_stream(ctx, sid)
    assert got == oracle.mine(ty, t, 16, I, theta, 3)
    L, E, iv = synth.level2_candidates(range(16), len(I))
    rel = oracle.count_batch(ty, t, L, E, iv, I, oracle.RELAXED)
    want = int((rel >= theta).sum())
    assert stats[0]["kernel_relaxed"] == fem.KERNEL_PAIRS and stats[0]["segments"] == 4
    assert want < stats[0]["survivors"] <= want + len(L) // 64


@pytest.fixture(scope="module")
def single_recording(ctx):
    cfg = synth.single_recording()
    s = cfg["stream"]
    sid = fem.fem_load_stream(ctx, s.types, s.t, s.n_types)
    return cfg, s, sid


def test_single_recording_level2_sampled(ctx, single_recording):
    """Full-size 64-type, 300 s recording: all 16,128 level-2 candidates counted in
    the bench's launch configuration; 256 sampled candidates checked one by one
    against the oracle, Theorem 5.1 checked on all."""
    cfg, s, sid = single_recording
    L, E, iv = synth.level2_candidates(range(64), 4)
    rec = fem.pack_episodes(L, E, iv)
    rel = fem.fem_count_candidates(ctx, sid, rec, cfg["intervals"], fem.PASS_RELAXED)
    ex = fem.fem_count_candidates(ctx, sid, rec, cfg["intervals"], fem.PASS_EXACT)
    assert np.all(rel >= ex)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(len(L), 256, replace=False))
    for p, got in ((oracle.RELAXED, rel), (oracle.EXACT, ex)):
        want = oracle.count_batch(s.types, s.t, L[pick], E[pick], iv[pick], cfg["intervals"], p)
        assert_counts_equal(got[pick], want, f"sampled pass {p}")


def test_single_recording_mining_sampled(ctx, single_recording):
    """Full-size mining at the workload threshold: every reported episode's count is
    re-derived by the oracle, every reported episode meets theta, and sampled level-2
    candidates missing from the result are below theta per the oracle."""
    cfg, s, sid = single_recording
    theta = cfg["theta"]
    got = fem.fem_mine_levelwise(ctx, sid, cfg["intervals"], theta, cfg["max_len"])
    for level, rows in got.items():
        if level == 1:
            continue
        keys = [oracle.canonical_key(r[0], r[1]) for r in rows]
        assert keys == sorted(keys)
        lens, E, iv = oracle._pack([(r[0], r[1]) for r in rows])
        want = oracle.count_batch(s.types, s.t, lens, E, iv, cfg["intervals"], oracle.EXACT)
        assert_counts_equal([r[2] for r in rows], want, f"level {level}")
        assert all(r[2] >= theta for r in rows)
    found2 = {(r[0], r[1]) for r in got.get(2, [])}
    L, E, iv = synth.level2_candidates(range(64), 4)
    rng = np.random.default_rng(1)
    pick = [i for i in rng.choice(len(L), 400, replace=False)
            if (tuple(E[i, :2]), (int(iv[i, 0]),)) not in found2][:200]
    pick = np.array(sorted(pick))
    want = oracle.count_batch(s.types, s.t, L[pick], E[pick], iv[pick], cfg["intervals"],
                              oracle.EXACT)
    assert np.all(want < theta)


def test_single_recording_deep_sampled(ctx):
    """The deep variant (theta = 300; about 12.5k frequent pairs, 2.4M level-3
    candidates): at every level the candidate count equals the oracle's join of the
    device's previous frequent set, sampled reported episodes have the oracle's exact
    count, and sampled candidates not reported are below theta per the oracle."""
    cfg = synth.single_recording(deep=True)
    s = cfg["stream"]
    I, theta = cfg["intervals"], cfg["theta"]
    sid = fem.fem_load_stream(ctx, s.types, s.t, s.n_types)
    got = fem.fem_mine_levelwise(ctx, sid, I, theta, cfg["max_len"])
    stats = fem.fem_last_mine_stats(ctx)
    fem.fem_free_stream(ctx, sid)
    assert max(got) >= 3 and stats[1]["candidates"] > 1_000_000
    rng = np.random.default_rng(7)
    for st in stats:
        N = st["level"]
        rows = got.get(N, [])
        assert st["frequent"] == len(rows)
        if N == 2:
            ft = [r[0][0] for r in got[1]]
            L, E, iv = synth.level2_candidates(ft, len(I))
            cands = [((int(E[i, 0]), int(E[i, 1])), (int(iv[i, 0]),)) for i in range(len(L))]
        else:
            cands = oracle.join([(r[0], r[1]) for r in got[N - 1]])
        assert len(cands) == st["candidates"], f"level {N} candidates"
        reported = {(r[0], r[1]): r[2] for r in rows}
        if rows:
            sel = [rows[i] for i in rng.choice(len(rows), min(48, len(rows)), replace=False)]
            lens, E, iv = oracle._pack([(r[0], r[1]) for r in sel])
            want = oracle.count_batch(s.types, s.t, lens, E, iv, I, oracle.EXACT)
            assert_counts_equal([r[2] for r in sel], want, f"level {N} reported")
        pool = [cands[i] for i in rng.choice(len(cands), min(400, len(cands)), replace=False)]
        absent = [c for c in pool if c not in reported][:48]
        if absent:
            lens, E, iv = oracle._pack(absent)
            want = oracle.count_batch(s.types, s.t, lens, E, iv, I, oracle.EXACT)
            assert np.all(want < theta), f"level {N} missing a frequent episode"


def test_large_stream_two_pass_sampled(ctx):
    """One hour at 50 Hz x 64 types (11.5M events), 100k candidates: Algorithm 4 on the
    device (autotuned mapping and one segment per chunk agree); 24 sampled candidates
    checked against the oracle, Theorem 5.1 on all."""
    torch = pytest.importorskip("torch")
    cfg = synth.large_stream()
    s = cfg["stream"]
    I, theta = cfg["intervals"], cfg["theta"]
    L, E, iv = cfg["candidates"]
    sid = fem.fem_load_stream(ctx, s.types, s.t, s.n_types)
    rec = torch.from_numpy(fem.pack_episodes(L, E, iv)).cuda()
    rel = torch.zeros(len(L), dtype=torch.int32, device="cuda")
    fem.fem_count_candidates(ctx, sid, rec, I, fem.PASS_RELAXED, out=rel)
    ex, sv = fem.fem_count_two_pass(ctx, sid, rec.cpu().numpy(), I, theta)
    fem.fem_set_config(ctx, segments=(s.n + 2047) // 2048)
    ex2, sv2 = fem.fem_count_two_pass(ctx, sid, rec.cpu().numpy(), I, theta)
    assert_counts_equal(ex2, ex, "one segment per chunk")
    assert_counts_equal(sv2, sv, "one segment per chunk survived")
    rel = rel.cpu().numpy().view(np.uint32)
    assert np.all((rel >= theta) == (sv != 0))
    rng = np.random.default_rng(3)
    surv = np.nonzero(sv)[0]
    pick = np.concatenate([rng.choice(len(L), 20, replace=False), surv[:4]]).astype(np.int64)
    want_r = oracle.count_batch(s.types, s.t, L[pick], E[pick], iv[pick], I, oracle.RELAXED)
    want_e = oracle.count_batch(s.types, s.t, L[pick], E[pick], iv[pick], I, oracle.EXACT)
    assert_counts_equal(rel[pick], want_r, "sampled relaxed")
    assert np.all(want_r >= want_e)
    for j, c in enumerate(pick):
        if sv[c]:
            assert ex[c] == want_e[j]
    fem.fem_free_stream(ctx, sid)
