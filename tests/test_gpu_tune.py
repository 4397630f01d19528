"""Measured mapping choice (the tuning cache that replaces the fixed crossover rule of
Algorithm 2): tuned counts equal the oracle, the cache round-trips through its JSON
file, and a cached shape is the one a later count uses."""
import json
import math

import numpy as np
import pytest

import oracle
from paper_0905_2200_gb300 import fem, synth
from tests.gpu_common import I_MS4, assert_counts_equal, ctx_fixture, mid_stream, mining_stream

pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    c = ctx_fixture()
    yield c
    fem.fem_destroy(c)


def oracle_counts(ty, t, L, E, iv, I, pass_):
    return oracle.count_batch(ty, t, L, E, iv, I, oracle.EXACT if pass_ else oracle.RELAXED)


def test_tuned_counts_equal_oracle_and_cache_round_trips(ctx, tmp_path):
    ty, t, K, _ = mid_stream()
    sid = fem.fem_load_stream(ctx, ty, t, K)
    L, E, iv = synth.level2_candidates(range(K), 4)
    rec = fem.pack_episodes(L, E, iv)
    fem.fem_tune_enable(ctx, True)
    for pass_ in (fem.PASS_RELAXED, fem.PASS_EXACT):
        got = fem.fem_count_candidates(ctx, sid, rec, I_MS4, pass_)
        assert_counts_equal(got, oracle_counts(ty, t, L, E, iv, I_MS4, pass_), f"tuned {pass_}")
        again = fem.fem_count_candidates(ctx, sid, rec, I_MS4, pass_)   # from the cache
        assert_counts_equal(again, got, "cached shape")
    assert fem.fem_tune_size(ctx) == 2
    path = tmp_path / "tune.jsonl"
    fem.fem_tune_save(ctx, path)
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) == 2 and all(x["segments"] >= 1 and x["threads"] >= 8 for x in lines)
    c2 = ctx_fixture()
    try:
        fem.fem_tune_load(c2, path)
        assert fem.fem_tune_size(c2) == 2
    finally:
        fem.fem_destroy(c2)


def test_cached_shape_is_used(ctx, tmp_path):
    """A cache entry written by hand for the level-2 relaxed class of this stream makes
    the miner run that pass with the entry's segment count, with the same result."""
    ty, t, K, _ = mining_stream()
    sid = fem.fem_load_stream(ctx, ty, t, K)
    theta = 80
    f1 = int((np.bincount(ty, minlength=K) >= theta).sum())
    m2 = f1 * (f1 - 1) * len(I_MS4)
    chunks = (len(t) + 2047) // 2048
    key = f"2/0/1/{math.ceil(math.log2(m2))}/{math.ceil(math.log2(chunks))}/{K}"
    path = tmp_path / "tune.jsonl"
    path.write_text(json.dumps({"key": key, "segments": 3, "threads": 64, "ms": 0.0}) + "\n")
    fem.fem_tune_load(ctx, path)
    got = fem.fem_mine_levelwise(ctx, sid, I_MS4, theta, 6)
    st = fem.fem_last_mine_stats(ctx)
    assert st[0]["level"] == 2 and st[0]["candidates"] == m2
    assert st[0]["segments"] == 3
    assert got == oracle.mine(ty, t, K, I_MS4, theta, 6)


def test_bad_cache_files_are_rejected(ctx, tmp_path):
    bad = tmp_path / "bad.jsonl"
    bad.write_text('{"key": "2/0/1/14/8/64", "segments": 0, "threads": 64, "ms": 0}\n')
    with pytest.raises(fem.FemError) as e:
        fem.fem_tune_load(ctx, bad)
    assert e.value.status == -1
    assert fem.fem_tune_size(ctx) == 0
    with pytest.raises(fem.FemError) as e:
        fem.fem_tune_load(ctx, tmp_path / "missing.jsonl")
    assert e.value.status == -11
