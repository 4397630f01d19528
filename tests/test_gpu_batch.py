"""Batched two-pass counting (many recordings, one persistent launch per pass per
episode length, replayed from a CUDA graph) against the single-recording path and
the oracle."""
import numpy as np
import pytest

import oracle
from paper_0905_2200_gb300 import fem, synth
from tests.gpu_common import assert_counts_equal, ctx_fixture

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = ctx_fixture()
    yield c
    fem.fem_destroy(c)


def make_jobs(ctx, batch, torch):
    jobs, meta = [], []
    for r, rec in enumerate(batch["recordings"]):
        s = rec["stream"]
        sid = fem.fem_load_stream(ctx, s.types, s.t, s.n_types)
        L, E, iv = rec["candidates"]
        for N in sorted(set(int(x) for x in L)):
            sel = np.nonzero(L == N)[0]
            recs = fem.pack_episodes(L[sel], E[sel], iv[sel])
            jobs.append(dict(stream_id=sid, len=N, theta=rec["theta"],
                             cands=torch.from_numpy(recs).cuda(),
                             exact_out=torch.full((len(sel),), 7, dtype=torch.int32, device="cuda"),
                             survived_out=torch.full((len(sel),), 7, dtype=torch.uint8,
                                                     device="cuda")))
            meta.append((r, sel))
    return jobs, meta


@pytest.mark.parametrize("tune", [False, True])
def test_batch_equals_single_recording_path_and_oracle(ctx, tune):
    """With tuning on, fem_batch_create first times every segment length / block size
    pair per length group (each a complete count) and captures the fastest."""
    torch = pytest.importorskip("torch")
    fem.fem_tune_enable(ctx, tune)
    batch = synth.batched_recordings(seed=0xB7, n_rec=10, t_range=(5.0, 150.0),
                                     m_range=(40, 1500))
    I = batch["intervals"]
    jobs, meta = make_jobs(ctx, batch, torch)
    b = fem.fem_batch_create(ctx, jobs, I)
    try:
        first = [(j["exact_out"].cpu().numpy().view(np.uint32).copy(),
                  j["survived_out"].cpu().numpy().copy()) for j in jobs]
        for j in jobs:  # the graph replay must rewrite every output
            j["exact_out"].fill_(7)
            j["survived_out"].fill_(7)
        fem.fem_batch_run(b)
        torch.cuda.synchronize()
        n_surv = 0
        for k, j in enumerate(jobs):
            ex = j["exact_out"].cpu().numpy().view(np.uint32)
            sv = j["survived_out"].cpu().numpy()
            assert_counts_equal(ex, first[k][0], f"job {k} replay exact")
            assert_counts_equal(sv, first[k][1], f"job {k} replay survived")
            ex1, sv1 = fem.fem_count_two_pass(ctx, j["stream_id"], j["cands"].cpu().numpy(), I,
                                              j["theta"])
            assert_counts_equal(sv, sv1, f"job {k} survived vs single")
            assert_counts_equal(ex, ex1, f"job {k} exact vs single")
            n_surv += int(sv.sum())
        assert n_surv > 0
        # oracle on a few jobs
        for k in range(0, len(jobs), max(1, len(jobs) // 6)):
            r, sel = meta[k]
            rec = batch["recordings"][r]
            s = rec["stream"]
            L, E, iv = rec["candidates"]
            _, ex_o, sv_o = oracle.two_pass(s.types, s.t, L[sel], E[sel], iv[sel], I, rec["theta"])
            assert_counts_equal(jobs[k]["survived_out"].cpu().numpy(), sv_o, f"job {k} oracle sv")
            assert_counts_equal(jobs[k]["exact_out"].cpu().numpy().view(np.uint32), ex_o,
                                f"job {k} oracle ex")
    finally:
        fem.fem_batch_destroy(b)
        fem.fem_tune_enable(ctx, False)
