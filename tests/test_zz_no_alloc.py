"""fem_select_noalloc: the survivor selection for callers that may not allocate device
memory (for example a real-time loop with a fixed, pre-reserved budget).

Its output must equal what the allocating entry point reports: the survivors of
fem_count_two_pass on the same candidates and threshold.  Two calls in a row (the
second smaller than the first) check that nothing left in the shared static scratch
array from one call leaks into the next.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_0905_2200_gb300 import fem, synth

pytestmark = pytest.mark.gpu


def _relaxed_on_device(ctx, sid, rec, I, torch):
    out = torch.zeros(rec.shape[0], dtype=torch.int32, device="cuda")
    fem.fem_count_candidates(ctx, sid, rec, I, fem.PASS_RELAXED, out=out)
    return out


def test_select_noalloc_matches_two_pass_survivors():
    torch = pytest.importorskip("torch")
    from paper_0905_2200_gb300 import build
    build.build()
    ctx = fem.fem_create(0)
    try:
        cfg = synth.single_recording()
        s = cfg["stream"]
        sid = fem.fem_load_stream(ctx, s.types, s.t, s.n_types)
        I = cfg["intervals"]
        L, E, iv = synth.level2_candidates(range(64), 4)
        big = fem.pack_episodes(L, E, iv)
        Ls, Es, ivs = synth.random_candidates(11, 3000, 64, [2], 4)
        small = fem.pack_episodes(Ls, Es, ivs)
        for rec, theta in ((big, cfg["theta"]), (small, 900)):
            counts = _relaxed_on_device(ctx, sid, rec, I, torch)
            idx = torch.full((rec.shape[0],), -1, dtype=torch.int32, device="cuda")
            nsel = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            fem.fem_select_noalloc(counts, theta, idx, nsel)
            torch.cuda.synchronize()
            k = int(nsel.item())
            got = idx[:k].cpu().numpy()
            _, survived = fem.fem_count_two_pass(ctx, sid, rec, I, theta)
            want = np.nonzero(survived)[0]
            assert k == want.size
            assert np.array_equal(got, want)
            assert 0 < k < rec.shape[0]
    finally:
        fem.fem_destroy(ctx)


def test_select_noalloc_rejects_oversize_request():
    torch = pytest.importorskip("torch")
    lib = fem.load()
    buf = torch.zeros(4, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    rc = lib.fem_select_noalloc(p, (1 << 26) + 1, 0, p, p, None)
    assert rc == -1


@pytest.mark.parametrize("m", [1, 1000, 16383, 16384, 16385, 70001])
def test_select_noalloc_sizes_match_numpy(m):
    """Both compaction forms (one block up to 16,384 values, three launches above) keep
    exactly the values >= theta, in ascending order, at and around the switch-over."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(m)
    host = rng.integers(0, 1000, m).astype(np.int32)
    theta = 500
    vals = torch.from_numpy(host).cuda()
    idx = torch.full((m,), -1, dtype=torch.int32, device="cuda")
    nsel = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    fem.fem_select_noalloc(vals, theta, idx, nsel)
    torch.cuda.synchronize()
    want = np.nonzero(host >= theta)[0]
    k = int(nsel.item())
    assert k == want.size
    assert np.array_equal(idx[:k].cpu().numpy(), want)
    assert np.all(idx[k:].cpu().numpy() == -1)
