"""The level-2 pair kernel (fem_count_pairs_relaxed: the relaxed pass over a complete
level-2 candidate set): one thread counts every interval variant of an ordered type pair.  Its
relaxed counts equal the oracle's (Algorithm 3, Section 5.3.1) element by element, with
one segment and with MapConcatenate segments (Section 5.2.2), on the benchmark recording
(the stored oracle counts of all 16,128 level-2 candidates), a mid-size stream, a
bursting recording (entry-class overflows recounted) and type lists in any order."""
import os

import numpy as np
import pytest

import oracle
from paper_0905_2200_gb300 import fem, synth
from tests.gpu_common import I_MS4, assert_counts_equal, ctx_fixture, mid_stream

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full")


@pytest.fixture(scope="module")
def ctx():
    c = ctx_fixture()
    yield c
    fem.fem_destroy(c)


@pytest.fixture(autouse=True)
def _reset(ctx):
    fem.fem_set_config(ctx, reset=True)
    yield
    fem.fem_set_config(ctx, reset=True)


def oracle_pairs(ty, t, types, I):
    L, E, iv = synth.level2_candidates(types, len(I))
    return oracle.count_batch(ty, t, L, E, iv, I, oracle.RELAXED)


@pytest.mark.parametrize("segments", [0, 1, 2, 7, 19])
@pytest.mark.parametrize("nI", [1, 3, 4])
def test_pairs_equal_oracle_mid_stream(ctx, segments, nI):
    ty, t, K, _ = mid_stream()
    sid = fem.fem_load_stream(ctx, ty, t, K)
    rng = np.random.default_rng(segments * 10 + nI)
    types = [int(x) for x in rng.permutation(K)[:20]]  # any order, a subset
    I = I_MS4[:nI] if nI < 4 else I_MS4
    fem.fem_set_config(ctx, segments=segments)
    got = fem.fem_count_pairs_relaxed(ctx, sid, types, I)
    assert_counts_equal(got, oracle_pairs(ty, t, types, I), f"P={segments} nI={nI}")
    fem.fem_free_stream(ctx, sid)


def test_pairs_benchmark_recording_full(ctx):
    """All 64 x 63 x 4 level-2 candidates of the benchmark recording against the stored
    oracle counts, with the rule's segments and with one segment."""
    cfg = synth.single_recording()
    s = cfg["stream"]
    d = np.load(os.path.join(GOLD, "single_recording.npz"))
    sid = fem.fem_load_stream(ctx, s.types, s.t, s.n_types)
    for seg in (0, 1):
        fem.fem_set_config(ctx, segments=seg)
        got = fem.fem_count_pairs_relaxed(ctx, sid, list(range(64)), cfg["intervals"])
        assert_counts_equal(got, d["L2_all_relaxed"], f"benchmark recording P={seg}")
    fem.fem_free_stream(ctx, sid)


def test_pairs_bursting_recording(ctx):
    """Bursts: windows hold more capable events than a variant's four class slots, so
    some candidates are recounted; every count still equals the oracle's."""
    cfg = synth.bursty_recording()
    s = cfg["stream"]
    sid = fem.fem_load_stream(ctx, s.types, s.t, s.n_types)
    types = list(range(0, 64, 4))
    for seg in (0, 40):
        fem.fem_set_config(ctx, segments=seg)
        got = fem.fem_count_pairs_relaxed(ctx, sid, types, cfg["intervals"])
        assert_counts_equal(got, oracle_pairs(s.types, s.t, types, cfg["intervals"]),
                            f"bursts P={seg}")
    fem.fem_free_stream(ctx, sid)


def test_pairs_argument_errors(ctx):
    ty, t, K, _ = mid_stream(seed=0xFA1, T=10.0)
    sid = fem.fem_load_stream(ctx, ty, t, K)
    for types, I in (([1, 2, 1], I_MS4),        # a repeated type
                     ([3], I_MS4),               # fewer than two types
                     ([1, K], I_MS4),            # a type out of range
                     ([1, 2], np.concatenate([I_MS4, I_MS4[:1]]))):  # five intervals
        with pytest.raises(fem.FemError) as e:
            fem.fem_count_pairs_relaxed(ctx, sid, types, I)
        assert e.value.status == -1
    fem.fem_free_stream(ctx, sid)
