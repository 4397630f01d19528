"""The C ABI library builds, loads and exports every entry point its header declares
(no GPU needed; no compute call is made)."""
import os
import re
import shutil
import subprocess

import pytest

from paper_0905_2200_gb300 import build as fembuild
from paper_0905_2200_gb300 import fem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fem.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fem_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    if shutil.which(fembuild.nvcc()) is None and not os.path.exists(fembuild.nvcc()):
        pytest.skip("nvcc not available")
    return fembuild.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("fem_load_stream", "fem_count_candidates", "fem_mine_levelwise",
                 "fem_count_two_pass", "fem_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib_path]).decode()
    exported = set(re.findall(r"\bT (fem_[a-z_0-9]+)$", out, flags=re.M))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_every_declared_symbol(lib_path):
    lib = fem.load(lib_path)
    for s in declared_symbols():
        assert hasattr(lib, s)
        assert s in fem.EXPORTS


def test_strerror_names_statuses(lib_path):
    fem.load(lib_path)
    assert fem.fem_strerror(0) == "ok"
    assert "sorted" in fem.fem_strerror(-2) or "decreasing" in fem.fem_strerror(-2)


def test_episode_record_layout():
    rec = fem.pack_episodes([3], [[1, 2, 3, 0, 0, 0, 0, 0]], [[0, 1, 0, 0, 0, 0, 0]])
    assert rec.shape == (1, 16)
    assert list(rec[0]) == [1, 2, 3, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 3]
    L, E, iv = fem.unpack_episodes(rec)
    assert L[0] == 3 and list(E[0, :3]) == [1, 2, 3] and list(iv[0, :2]) == [0, 1]


def test_interval_marshalling():
    """Interval sets reach the C ABI as fem_interval records in the given order (lists,
    uint32 arrays, non-contiguous views, and the empty set)."""
    import numpy as np
    want = [(0, 2000), (2000, 5000), (5000, 10000), (10000, 20000)]
    arr = np.array(want, np.uint32)
    for given in (want, arr, np.asfortranarray(arr), arr[::-1][::-1]):
        recs, n = fem._intervals(given)
        assert n == 4
        assert [(recs[i].lo_us, recs[i].hi_us) for i in range(n)] == want
    recs, n = fem._intervals(np.zeros((0, 2), np.uint32))
    assert n == 0
