"""Level-wise generation with more frequent episodes than the join's one-block scan and
shared-memory staging take (19,460 frequent pairs): the join places every child, the
level-3 candidate count equals the join of the device's frequent pairs, and sampled
level-3 episodes agree with the oracle."""
import numpy as np
import pytest

import oracle
from paper_0905_2200_gb300 import fem
from tests.gpu_common import assert_counts_equal, ctx_fixture

pytestmark = pytest.mark.gpu


def test_join_past_one_block_scan():
    K, R = 140, 30
    rng = np.random.default_rng(5)
    # rounds of all K types in random order, 7 us apart: every ordered pair of distinct
    # types occurs within 2 ms about once per round
    types = np.concatenate([rng.permutation(K) for _ in range(R)]).astype(np.uint8)
    t = (np.arange(types.size, dtype=np.uint32) * 7).astype(np.uint32)
    I = np.array([[0, 2000]], np.uint32)
    theta = 3
    ctx = ctx_fixture()
    try:
        sid = fem.fem_load_stream(ctx, types, t, K)
        got = fem.fem_mine_levelwise(ctx, sid, I, theta, 3, raw=True)
        stats = fem.fem_last_mine_stats(ctx)
    finally:
        fem.fem_destroy(ctx)
    rec2, cnt2 = got[2]
    f2 = rec2.shape[0]
    assert f2 > 16384, "the test needs a frequent set past the one-block scan"
    assert stats[0]["candidates"] == K * (K - 1)
    # the join of the device's frequent pairs: alpha (a, b) takes every (b, c), c != a
    a2, b2 = rec2[:, 0].astype(np.int64), rec2[:, 1].astype(np.int64)
    present = np.zeros((K, K), bool)
    present[a2, b2] = True
    outdeg = present.sum(axis=1)
    want_m3 = int(np.sum(outdeg[b2] - present[b2, a2]))
    assert stats[1]["candidates"] == want_m3
    # level-2 counts, sampled
    pick = np.sort(rng.choice(f2, 64, replace=False))
    lens = np.full(pick.size, 2, np.uint8)
    E = np.zeros((pick.size, 8), np.uint8)
    E[:, :2] = rec2[pick, :2]
    iv = np.zeros((pick.size, 7), np.uint8)
    want = oracle.count_batch(types, t, lens, E, iv, I, oracle.EXACT)
    assert_counts_equal(cnt2[pick], want, "level 2")
    # level 3: canonical (ascending) order, and sampled children of the join are
    # reported exactly when the oracle finds them frequent, with its count
    rec3, cnt3 = got.get(3, (np.zeros((0, 16), np.uint8), np.zeros(0, np.uint32)))
    code3 = (rec3[:, 0].astype(np.int64) * K + rec3[:, 1]) * K + rec3[:, 2]
    assert np.all(np.diff(code3) > 0)
    assert stats[1]["frequent"] == rec3.shape[0]
    al = rng.choice(f2, 96)
    kids = []
    for i in al:
        cs = np.nonzero(present[b2[i]])[0]
        cs = cs[cs != a2[i]]
        kids.append((int(a2[i]), int(b2[i]), int(rng.choice(cs))))
    lens = np.full(len(kids), 3, np.uint8)
    E = np.zeros((len(kids), 8), np.uint8)
    E[:, :3] = np.array(kids, np.uint8)
    iv = np.zeros((len(kids), 7), np.uint8)
    want = oracle.count_batch(types, t, lens, E, iv, I, oracle.EXACT)
    codes = (E[:, 0].astype(np.int64) * K + E[:, 1]) * K + E[:, 2]
    pos = np.searchsorted(code3, codes)
    hit = (pos < code3.size) & (code3[np.minimum(pos, code3.size - 1)] == codes)
    assert np.array_equal(hit, want >= theta)
    assert_counts_equal(cnt3[pos[hit]], want[hit], "level 3")
