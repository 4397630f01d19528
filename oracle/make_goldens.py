"""Writes the stored expected results of the full-size workloads (TEST INFRASTRUCTURE).

    python -m oracle.make_goldens [name ...] [--procs P]

Each file ``tests/golden/full/<name>.npz`` holds what the oracle computes for one
workload of ``paper_0905_2200_gb300.synth``, plus the SHA-256 of the generated inputs
it was computed from (``inputs_sha256``; the GPU tests regenerate the inputs, check
the digest, and compare the CUDA results element by element with these arrays).
Nothing here reads the CUDA library: every value comes from ``oracle`` (the plain
single-threaded counters of ``fem_oracle.c``, run as independent processes over
candidate shards by ``oracle.shards``).

Workloads and contents:
  tiny_mining          Problem 1 mined to length 4 (every level's frequent set).
  single_recording     mined to length 6; all 16,128 level-2 candidates' relaxed
                       (Algorithm 3) and exact (Algorithm 1) counts; the level-3
                       candidates (join of the frequent pairs): Algorithm 4's
                       relaxed, exact-if-survived and survived arrays.
  single_recording_deep  theta 300: mined to length 6; level-3 candidates (about
                       2.4M) through Algorithm 4 as above.
  large_stream         100,000 candidates over the 11.8M-event hour: Algorithm 4.
  batched              256 recordings, one job per (recording, length): Algorithm 4
                       per job, concatenated in job order (recordings in order,
                       lengths ascending), with the job offsets.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle.shards import ShardPool, two_pass_jobs  # noqa: E402
from paper_0905_2200_gb300 import synth  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "full")


def mined_arrays(res, max_len):
    """{level: rows} -> flat arrays L<k>_types / L<k>_ivl / L<k>_counts per level."""
    out = {}
    for k in range(1, max_len + 1):
        rows = res.get(k, [])
        ty = np.zeros((len(rows), oracle.LMAX), np.uint8)
        iv = np.zeros((len(rows), oracle.LMAX - 1), np.uint8)
        cn = np.zeros(len(rows), np.uint32)
        for i, (a, b, c) in enumerate(rows):
            ty[i, :len(a)] = a
            iv[i, :len(b)] = b
            cn[i] = c
        out[f"L{k}_types"], out[f"L{k}_ivl"], out[f"L{k}_counts"] = ty, iv, cn
    return out


def stream_digest(cfg, extra=()):
    s = cfg["stream"]
    return synth.digest(s.types, s.t, cfg["intervals"], np.array([cfg["theta"]]), *extra)


def save(name, **arrays):
    os.makedirs(OUT, exist_ok=True)
    path = os.path.join(OUT, name + ".npz")
    np.savez_compressed(path, **arrays)
    print(f"wrote {path} ({os.path.getsize(path) / 1e6:.2f} MB)", flush=True)


def w_tiny(procs):
    cfg = synth.tiny_mining()
    s = cfg["stream"]
    with ShardPool(s.types, s.t, procs) as pool:
        res = oracle.mine(s.types, s.t, s.n_types, cfg["intervals"], cfg["theta"],
                          cfg["max_len"], counter=pool)
    save("tiny_mining", inputs_sha256=np.array(stream_digest(cfg)),
         **mined_arrays(res, cfg["max_len"]))


def _level3(res, with_pool, I, theta):
    c3 = oracle.join([(r[0], r[1]) for r in res[2]])
    L3, E3, iv3 = oracle._pack(c3)
    return (L3, E3, iv3), with_pool.two_pass(L3, E3, iv3, I, theta)


def w_single(procs, deep=False):
    cfg = synth.single_recording(deep=deep)
    s, I, theta = cfg["stream"], cfg["intervals"], cfg["theta"]
    L2, E2, iv2 = synth.level2_candidates(range(64), len(I))
    with ShardPool(s.types, s.t, procs) as pool:
        res = oracle.mine(s.types, s.t, s.n_types, I, theta, cfg["max_len"], counter=pool)
        arrays = mined_arrays(res, cfg["max_len"])
        if not deep:
            arrays["L2_all_relaxed"] = pool.count_batch(L2, E2, iv2, I, oracle.RELAXED)
            arrays["L2_all_exact"] = pool.count_batch(L2, E2, iv2, I, oracle.EXACT)
        (L3, E3, iv3), (rel, ex, sv) = _level3(res, pool, I, theta)
    arrays["L3_cands_sha256"] = np.array(synth.digest(L3, E3, iv3))
    arrays["L3_relaxed"], arrays["L3_exact"], arrays["L3_survived"] = rel, ex, sv
    save("single_recording" + ("_deep" if deep else ""),
         inputs_sha256=np.array(stream_digest(cfg)), **arrays)


def w_large(procs):
    cfg = synth.large_stream()
    s, I, theta = cfg["stream"], cfg["intervals"], cfg["theta"]
    L, E, iv = cfg["candidates"]
    with ShardPool(s.types, s.t, procs) as pool:
        rel, ex, sv = pool.two_pass(L, E, iv, I, theta)
    save("large_stream", inputs_sha256=np.array(stream_digest(cfg, (L, E, iv))),
         relaxed=rel, exact=ex, survived=sv)


def batched_jobs(batch):
    """(recording index, length, candidate selection) per job, in job order."""
    out = []
    for r, rec in enumerate(batch["recordings"]):
        L = rec["candidates"][0]
        for N in sorted(set(int(x) for x in L)):
            out.append((r, N, np.nonzero(L == N)[0]))
    return out


def batched_digest(batch):
    parts = [batch["intervals"]]
    for rec in batch["recordings"]:
        s = rec["stream"]
        parts += [s.types, s.t, np.array([rec["theta"]]), *rec["candidates"]]
    return synth.digest(*parts)


def w_batched(procs):
    batch = synth.batched_recordings()
    I = batch["intervals"]
    jobs = batched_jobs(batch)
    args = []
    for r, N, sel in jobs:
        rec = batch["recordings"][r]
        s = rec["stream"]
        L, E, iv = rec["candidates"]
        args.append((s.types, s.t, L[sel], E[sel], iv[sel], I, rec["theta"]))
    # longest jobs first over the pool, results put back in job order
    cost = [len(a[2]) * len(a[1]) for a in args]
    order = np.argsort(cost)[::-1]
    res = two_pass_jobs([args[i] for i in order], procs)
    out = [None] * len(args)
    for i, r in zip(order, res):
        out[i] = r
    off = np.zeros(len(jobs) + 1, np.int64)
    off[1:] = np.cumsum([len(sel) for _, _, sel in jobs])
    save("batched", inputs_sha256=np.array(batched_digest(batch)), job_offsets=off,
         job_recording=np.array([r for r, _, _ in jobs], np.int32),
         job_length=np.array([N for _, N, _ in jobs], np.int32),
         relaxed=np.concatenate([o[0] for o in out]), exact=np.concatenate([o[1] for o in out]),
         survived=np.concatenate([o[2] for o in out]))


WRITERS = {
    "tiny_mining": w_tiny,
    "single_recording": w_single,
    "single_recording_deep": lambda p: w_single(p, deep=True),
    "large_stream": w_large,
    "batched": w_batched,
}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("names", nargs="*", default=list(WRITERS))
    ap.add_argument("--procs", type=int, default=0, help="oracle processes (default: all cores)")
    a = ap.parse_args(argv)
    for name in a.names:
        t0 = time.time()
        WRITERS[name](a.procs or None)
        print(f"{name}: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
