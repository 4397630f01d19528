"""Serving: streams that grow chunk by chunk, one-shot and standing requests admitted
while others run (continuous batching).  Each result must equal the oracle on the
event range it covers, and must be the same when the request runs alone as when it
runs in the mix."""
import numpy as np
import pytest

import oracle
from paper_0905_2200_gb300 import fem, synth
from tests.gpu_common import I_MS4, assert_counts_equal, ctx_fixture

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = ctx_fixture()
    yield c
    fem.fem_destroy(c)


def live_streams(n=3, T=40.0):
    out = []
    for k in range(n):
        K = [20, 32, 48][k % 3]
        rng = np.random.default_rng(100 + k)
        ch = []
        for L in (3, 4):
            tys = tuple(int(x) for x in rng.choice(K, L, replace=False))
            ivs = tuple(int(x) for x in rng.integers(0, 4, L - 1))
            ch.append((tys, 4.0, [tuple(I_MS4[i]) for i in ivs]))
        t, ty = synth.poisson_stream(500 + k, K, float(rng.uniform(10, 40)), T, chains=ch)
        out.append((ty, t, K, ch))
    return out


def chunks_of(t, dt_us=100_000):
    edges = np.searchsorted(t, np.arange(0, int(t[-1]) + dt_us + 1, dt_us))
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:])]


def request_set(seed, K, m):
    L, E, iv = synth.random_candidates(seed, m, K, [2, 3, 4], 4)
    return L, E, iv, fem.pack_episodes(L, E, iv)


def run_scenario(ctx, streams, plan, chunk_every=5):
    """Feed the streams chunk by chunk; submit plan[(step, stream, request)] at the given
    chunk step; poll every step.  Returns {name: (counts, flags, events, status, range)}."""
    srv = fem.fem_server_create(ctx, mem_budget_bytes=256 << 20, max_active=32, n_lanes=4)
    try:
        sids = [fem.fem_server_open_stream(srv, K, len(t) + 4096) for ty, t, K, ch in streams]
        cks = [chunks_of(t) for ty, t, K, ch in streams]
        fed = [0] * len(streams)
        names, ranges, res = {}, {}, {}
        steps = max(len(c) for c in cks)
        for step in range(steps):
            for i, (ty, t, K, ch) in enumerate(streams):
                if step < len(cks[i]):
                    a, b = cks[i][step]
                    if b > a:
                        fem.fem_server_append(srv, sids[i], ty[a:b], t[a:b])
                    fed[i] = b
            for (st, i, name, rec, theta, mode, win) in plan:
                if st == step:
                    rid = fem.fem_server_submit(srv, sids[i], rec, I_MS4, theta, mode, win)
                    names[rid] = name
                    ranges[name] = (i, fed[i], mode, win)
            fem.fem_server_poll(srv)
        fem.fem_server_drain(srv)
        for rid, nm in names.items():
            rec = next(p[3] for p in plan if p[2] == nm)
            c, f, ev, status = fem.fem_server_result(srv, rid, rec.shape[0])
            res[nm] = (c, f, ev, status, ranges[nm])
            fem.fem_server_release(srv, rid)
        return res
    finally:
        fem.fem_server_destroy(srv)


def test_serving_results_equal_oracle_and_alone_vs_mix(ctx):
    streams = live_streams()
    sets = {}
    plan = []
    for j, (step, i, mode, win) in enumerate([(60, 0, fem.REQ_ONESHOT, 5_000_000),
                                              (120, 1, fem.REQ_ONESHOT, 0),
                                              (150, 2, fem.REQ_ONESHOT, 12_000_000),
                                              (30, 0, fem.REQ_STANDING, 0),
                                              (200, 1, fem.REQ_STANDING, 0),
                                              (250, 2, fem.REQ_ONESHOT, 3_000_000)]):
        ty, t, K, ch = streams[i]
        L, E, iv, rec = request_set(900 + j, K, 300 + 150 * j)
        sets[f"r{j}"] = (L, E, iv)
        plan.append((step, i, f"r{j}", rec, 8 if mode == fem.REQ_ONESHOT else 0, mode, win))
    mix = run_scenario(ctx, streams, plan)
    for name, (c, f, ev, status, (i, fed, mode, win)) in mix.items():
        assert status == 0, name
        ty, t, K, ch = streams[i]
        L, E, iv = sets[name]
        if mode == fem.REQ_ONESHOT:
            end = fed
            begin = end - ev
            if win:
                assert t[begin] >= t[end - 1] - win and (begin == 0 or t[begin - 1] < t[end - 1] - win)
            theta = 8
            _, ex_o, sv_o = oracle.two_pass(ty[begin:end], t[begin:end], L, E, iv, I_MS4, theta)
            assert_counts_equal(f, sv_o, f"{name} survived")
            assert_counts_equal(c, ex_o, f"{name} exact")
        else:
            begin, end = fed, len(t)
            assert ev == end - begin
            want = oracle.count_batch(ty[begin:end], t[begin:end], L, E, iv, I_MS4, oracle.EXACT)
            assert_counts_equal(c, want, f"{name} standing")
    # the same requests alone (one at a time, same submission points)
    for p in plan:
        alone = run_scenario(ctx, streams, [p])
        a = alone[p[2]]
        b = mix[p[2]]
        assert a[2] == b[2] and a[3] == b[3]
        assert_counts_equal(a[0], b[0], f"{p[2]} alone vs mix counts")
        assert_counts_equal(a[1], b[1], f"{p[2]} alone vs mix flags")


def test_admission_by_memory(ctx):
    ty, t, K, ch = live_streams(1)[0]
    srv = fem.fem_server_create(ctx, mem_budget_bytes=4 << 20, max_active=8, n_lanes=2)
    try:
        sid = fem.fem_server_open_stream(srv, K, len(t))
        fem.fem_server_append(srv, sid, ty, t)
        _, _, _, big = request_set(1, K, 80_000)   # ~2.8 MB of device memory each
        r1 = fem.fem_server_submit(srv, sid, big, I_MS4, 5)
        with pytest.raises(fem.FemError) as e:
            fem.fem_server_submit(srv, sid, big, I_MS4, 5)
        assert e.value.status == -6
        fem.fem_server_drain(srv)
        c1 = fem.fem_server_result(srv, r1, big.shape[0])
        assert c1[3] == 0
        # the finished one-shot returned its device memory: the next one is admitted
        r2 = fem.fem_server_submit(srv, sid, big, I_MS4, 5)
        fem.fem_server_drain(srv)
        c2 = fem.fem_server_result(srv, r2, big.shape[0])
        assert_counts_equal(c2[0], c1[0], "same request twice")
    finally:
        fem.fem_server_destroy(srv)


def test_serving_32_stream_workload_equals_oracle(ctx):
    """The serving workload's configuration: 32 live streams (16-128 types, 10-100 Hz,
    embedded chains) fed in 100 ms chunks; one one-shot request per stream over its last
    5 s and eight standing requests, submitted while the others run.  Every result equals
    the oracle on the event range it covers."""
    raw = synth.serving_streams(seed=0xFE05, n_streams=32, duration_s=20.0)
    streams = [(x["stream"].types, x["stream"].t, x["stream"].n_types, None) for x in raw]
    plan, sets = [], {}
    for i, (ty, t, K, _) in enumerate(streams):
        L, E, iv, rec = request_set(0x3200 + i, K, 400)
        sets[f"o{i}"] = (L, E, iv)
        plan.append((100 + 2 * i, i, f"o{i}", rec, 8, fem.REQ_ONESHOT, 5_000_000))
    for k in range(8):
        i = 4 * k
        ty, t, K, _ = streams[i]
        L, E, iv, rec = request_set(0x3300 + k, K, 300)
        sets[f"s{k}"] = (L, E, iv)
        plan.append((60 + k, i, f"s{k}", rec, 0, fem.REQ_STANDING, 0))
    res = run_scenario(ctx, streams, plan)
    assert len(res) == len(plan)
    for name, (c, f, ev, status, (i, fed, mode, win)) in res.items():
        assert status == 0, name
        ty, t, K, _ = streams[i]
        L, E, iv = sets[name]
        if mode == fem.REQ_ONESHOT:
            end = fed
            begin = end - ev
            assert t[begin] >= t[end - 1] - win and (begin == 0 or t[begin - 1] < t[end - 1] - win)
            _, ex_o, sv_o = oracle.two_pass(ty[begin:end], t[begin:end], L, E, iv, I_MS4, 8)
            assert_counts_equal(f, sv_o, f"{name} survived")
            assert_counts_equal(c, ex_o, f"{name} exact")
        else:
            begin, end = fed, len(t)
            assert ev == end - begin
            want = oracle.count_batch(ty[begin:end], t[begin:end], L, E, iv, I_MS4, oracle.EXACT)
            assert_counts_equal(c, want, f"{name} standing")
