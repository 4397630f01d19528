"""Shared helpers for the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np

import oracle
from paper_0905_2200_gb300 import fem, synth

I_MS4 = synth.I_MS4


def ctx_fixture():
    from paper_0905_2200_gb300 import build as b
    b.build()
    ctx = fem.fem_create(0)
    return ctx


def mid_stream(seed=0xFE10, K=32, rate=20.0, T=60.0):
    """~38k events (19 chunks of 2048 plus a ragged tail) with 4 embedded chains."""
    rng = np.random.default_rng(seed)
    chains = []
    for _ in range(4):
        L = int(rng.integers(3, 6))
        tys = tuple(int(x) for x in rng.choice(K, L, replace=False))
        ivs = tuple(int(x) for x in rng.integers(0, 4, L - 1))
        chains.append((tys, float(rng.uniform(1, 3)), [tuple(I_MS4[i]) for i in ivs]))
    t, ty = synth.poisson_stream(seed, K, rate, T, chains=chains)
    return ty, t, K, chains


def mining_stream(seed=0xFE11, K=24, rate=10.0, T=60.0):
    """~19k events (10 chunks) with three strong chains (4-6 Hz, lengths 4-6), so that
    level-wise mining reaches length 6 while chance pairs stay below the thresholds
    the tests use."""
    rng = np.random.default_rng(seed)
    chains = []
    for L in (4, 5, 6):
        tys = tuple(int(x) for x in rng.choice(K, L, replace=False))
        ivs = tuple(int(x) for x in rng.integers(0, 4, L - 1))
        chains.append((tys, float(rng.uniform(4, 6)), [tuple(I_MS4[i]) for i in ivs]))
    t, ty = synth.poisson_stream(seed, K, rate, T, chains=chains)
    return ty, t, K, chains


def oracle_counts(ty, t, L, E, iv, I, pass_):
    return oracle.count_batch(ty, t, L, E, iv, I,
                              oracle.RELAXED if pass_ == fem.PASS_RELAXED else oracle.EXACT)


def assert_counts_equal(got, want, what=""):
    got = np.asarray(got)
    want = np.asarray(want)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, (f"{what}: {bad.size} of {got.size} differ; first "
                           f"{[(int(i), int(got[i]), int(want[i])) for i in bad[:5]]}")
