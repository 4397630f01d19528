"""Full-size parity: on the full-size workloads, every output of the CUDA path equals the
oracle's, element by element -- every mined level, every candidate's relaxed and exact
count, every survived flag, every batch job.

The expected arrays are stored in ``tests/golden/full/*.npz``, written by
``python -m oracle.make_goldens`` (the plain C oracle over candidate shards; nothing in
them comes from the CUDA path).  Each file records the SHA-256 of the generated inputs
it was computed from; the tests regenerate the inputs and check that digest first.
Paper basis: Problem 1 (Section 2), Algorithms 1 and 3 (Sections 5.1, 5.3.1),
Algorithm 4 and Theorem 5.1 (Section 5.3.2)."""
import os

import numpy as np
import pytest

import oracle
from oracle.make_goldens import batched_digest, batched_jobs
from paper_0905_2200_gb300 import fem, synth
from tests.gpu_common import assert_counts_equal, ctx_fixture

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full")


def golden(name, digest):
    d = dict(np.load(os.path.join(GOLD, name + ".npz")))
    assert str(d["inputs_sha256"]) == digest, (
        f"{name}: the generated inputs differ from those the stored results were computed "
        f"from (regenerate with python -m oracle.make_goldens {name})")
    return d


def stream_digest(cfg, extra=()):
    s = cfg["stream"]
    return synth.digest(s.types, s.t, cfg["intervals"], np.array([cfg["theta"]]), *extra)


@pytest.fixture(scope="module")
def ctx():
    c = ctx_fixture()
    yield c
    fem.fem_destroy(c)


@pytest.fixture(autouse=True)
def _reset(ctx):
    fem.fem_set_config(ctx, reset=True)
    fem.fem_tune_enable(ctx, False)
    yield
    fem.fem_set_config(ctx, reset=True)
    fem.fem_tune_enable(ctx, False)


def assert_mined_equal(got_raw, gold, max_len):
    """fem_mine_levelwise(raw=True) vs the stored frequent sets, level by level."""
    for k in range(1, max_len + 1):
        ty, iv, cn = gold[f"L{k}_types"], gold[f"L{k}_ivl"], gold[f"L{k}_counts"]
        rec, cnt = got_raw.get(k, (np.zeros((0, 16), np.uint8), np.zeros(0, np.uint32)))
        assert rec.shape[0] == ty.shape[0], f"level {k}: {rec.shape[0]} frequent, oracle {ty.shape[0]}"
        assert np.array_equal(rec[:, :8], ty), f"level {k}: episode types differ"
        assert np.array_equal(rec[:, 8:15], iv), f"level {k}: intervals differ"
        assert np.all(rec[:, 15] == k)
        assert_counts_equal(cnt, cn, f"level {k} counts")


def level3(gold):
    rows = [(tuple(int(x) for x in gold["L2_types"][i, :2]), (int(gold["L2_ivl"][i, 0]),))
            for i in range(gold["L2_types"].shape[0])]
    L3, E3, iv3 = oracle._pack(oracle.join(rows))
    assert synth.digest(L3, E3, iv3) == str(gold["L3_cands_sha256"])
    return L3, E3, iv3


def check_two_pass(ctx, sid, rec_dev, I, theta, rel_g, ex_g, sv_g, what):
    torch = pytest.importorskip("torch")
    m = rec_dev.shape[0]
    rel = torch.zeros(m, dtype=torch.int32, device="cuda")
    fem.fem_count_candidates(ctx, sid, rec_dev, I, fem.PASS_RELAXED, out=rel)
    assert_counts_equal(rel.cpu().numpy().view(np.uint32), rel_g, f"{what} relaxed")
    ex = torch.zeros(m, dtype=torch.int32, device="cuda")
    sv = torch.zeros(m, dtype=torch.uint8, device="cuda")
    fem.fem_count_two_pass(ctx, sid, rec_dev, I, theta, exact_out=ex, survived_out=sv)
    assert_counts_equal(sv.cpu().numpy(), sv_g, f"{what} survived")
    assert_counts_equal(ex.cpu().numpy().view(np.uint32), ex_g, f"{what} exact")


def test_tiny_mining_full(ctx):
    cfg = synth.tiny_mining()
    s = cfg["stream"]
    gold = golden("tiny_mining", stream_digest(cfg))
    sid = fem.fem_load_stream(ctx, s.types, s.t, s.n_types)
    got = fem.fem_mine_levelwise(ctx, sid, cfg["intervals"], cfg["theta"], cfg["max_len"], raw=True)
    assert_mined_equal(got, gold, cfg["max_len"])
    fem.fem_free_stream(ctx, sid)


@pytest.mark.parametrize("tune", [True, False])
def test_single_recording_full(ctx, tune):
    """The benchmark's workload (64 types, 300 s, theta 1177) in the benchmark's launch
    configuration (measured launch shapes) and with the occupancy rule: the mined sets at
    every level, all 16,128 level-2 candidates' relaxed and exact counts, and the
    level-3 candidates through Algorithm 4."""
    torch = pytest.importorskip("torch")
    cfg = synth.single_recording()
    s, I, theta = cfg["stream"], cfg["intervals"], cfg["theta"]
    gold = golden("single_recording", stream_digest(cfg))
    fem.fem_tune_enable(ctx, tune)
    d_ty = torch.from_numpy(s.types.copy()).cuda()
    d_t = torch.from_numpy(s.t.view(np.int32).copy()).cuda()
    sid = fem.fem_load_stream(ctx, d_ty, d_t, s.n_types)
    got = fem.fem_mine_levelwise(ctx, sid, I, theta, cfg["max_len"], raw=True)
    assert_mined_equal(got, gold, cfg["max_len"])
    L2, E2, iv2 = synth.level2_candidates(range(64), len(I))
    rec2 = torch.from_numpy(fem.pack_episodes(L2, E2, iv2)).cuda()
    for pass_, key in ((fem.PASS_RELAXED, "L2_all_relaxed"), (fem.PASS_EXACT, "L2_all_exact")):
        out = torch.zeros(rec2.shape[0], dtype=torch.int32, device="cuda")
        fem.fem_count_candidates(ctx, sid, rec2, I, pass_, out=out)
        assert_counts_equal(out.cpu().numpy().view(np.uint32), gold[key], key)
    L3, E3, iv3 = level3(gold)
    rec3 = torch.from_numpy(fem.pack_episodes(L3, E3, iv3)).cuda()
    check_two_pass(ctx, sid, rec3, I, theta, gold["L3_relaxed"], gold["L3_exact"],
                   gold["L3_survived"], "level 3")
    fem.fem_free_stream(ctx, sid)


def test_single_recording_deep_full(ctx):
    """theta = 300: about 12.5k frequent pairs and 2.4M level-3 candidates; the mined sets
    at every level and every level-3 candidate through Algorithm 4."""
    torch = pytest.importorskip("torch")
    cfg = synth.single_recording(deep=True)
    s, I, theta = cfg["stream"], cfg["intervals"], cfg["theta"]
    gold = golden("single_recording_deep", stream_digest(cfg))
    sid = fem.fem_load_stream(ctx, s.types, s.t, s.n_types)
    got = fem.fem_mine_levelwise(ctx, sid, I, theta, cfg["max_len"], raw=True)
    assert_mined_equal(got, gold, cfg["max_len"])
    L3, E3, iv3 = level3(gold)
    assert len(L3) > 1_000_000
    rec3 = torch.from_numpy(fem.pack_episodes(L3, E3, iv3)).cuda()
    check_two_pass(ctx, sid, rec3, I, theta, gold["L3_relaxed"], gold["L3_exact"],
                   gold["L3_survived"], "level 3")
    fem.fem_free_stream(ctx, sid)


def test_large_stream_full(ctx):
    """One hour at 50 Hz x 64 types (11.8M events), all 100,000 candidates: relaxed
    counts, survived flags and exact counts equal the oracle's, with the measured launch
    shapes and with one MapConcatenate segment per chunk (5,755 segments)."""
    torch = pytest.importorskip("torch")
    cfg = synth.large_stream()
    s, I, theta = cfg["stream"], cfg["intervals"], cfg["theta"]
    L, E, iv = cfg["candidates"]
    gold = golden("large_stream", stream_digest(cfg, (L, E, iv)))
    sid = fem.fem_load_stream(ctx, torch.from_numpy(s.types).cuda(),
                              torch.from_numpy(s.t.view(np.int32)).cuda(), s.n_types)
    rec = torch.from_numpy(fem.pack_episodes(L, E, iv)).cuda()
    fem.fem_tune_enable(ctx, True)
    check_two_pass(ctx, sid, rec, I, theta, gold["relaxed"], gold["exact"], gold["survived"],
                   "tuned")
    fem.fem_tune_enable(ctx, False)
    fem.fem_set_config(ctx, segments=(s.n + 2047) // 2048)
    check_two_pass(ctx, sid, rec, I, theta, gold["relaxed"], gold["exact"], gold["survived"],
                   "one segment per chunk")
    fem.fem_free_stream(ctx, sid)


def test_batched_full(ctx):
    """256 recordings (42.5M events), 1,792 jobs: the batched persistent form replayed
    from its CUDA graph equals the oracle on every job and candidate."""
    torch = pytest.importorskip("torch")
    batch = synth.batched_recordings()
    I = batch["intervals"]
    gold = golden("batched", batched_digest(batch))
    off = gold["job_offsets"]
    jobs = []
    sids = []
    for k, (r, N, sel) in enumerate(batched_jobs(batch)):
        rec = batch["recordings"][r]
        s = rec["stream"]
        if len(sids) <= r:
            sids.append(fem.fem_load_stream(ctx, s.types, s.t, s.n_types))
        L, E, iv = rec["candidates"]
        assert gold["job_recording"][k] == r and gold["job_length"][k] == N
        assert off[k + 1] - off[k] == len(sel)
        jobs.append(dict(stream_id=sids[r], len=N, theta=rec["theta"],
                         cands=torch.from_numpy(fem.pack_episodes(L[sel], E[sel], iv[sel])).cuda(),
                         exact_out=torch.full((len(sel),), 7, dtype=torch.int32, device="cuda"),
                         survived_out=torch.full((len(sel),), 7, dtype=torch.uint8,
                                                 device="cuda")))
    b = fem.fem_batch_create(ctx, jobs, I)
    try:
        for j in jobs:  # the replay must write every output
            j["exact_out"].fill_(7)
            j["survived_out"].fill_(7)
        fem.fem_batch_run(b)
        torch.cuda.synchronize()
        ex = np.concatenate([j["exact_out"].cpu().numpy().view(np.uint32) for j in jobs])
        sv = np.concatenate([j["survived_out"].cpu().numpy() for j in jobs])
        assert_counts_equal(sv, gold["survived"], "batched survived")
        assert_counts_equal(ex, gold["exact"], "batched exact")
    finally:
        fem.fem_batch_destroy(b)
        for sid in sids:
            fem.fem_free_stream(ctx, sid)
