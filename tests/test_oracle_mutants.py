"""The oracle's pins are sensitive: each plausible mistake planted in a copy of the
oracle's C source (a boundary of the (lo, hi] test, a dropped reset, a reversed
node order, a wrong MapConcatenate window, ...) makes the pin suite fail.  The
mistakes are planted on the CPU, in a temporary copy; the oracle itself is not
changed."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fem_oracle.c")

# (name, exact text in fem_oracle.c, planted replacement)
MUTANTS = [
    ("lists: lo bound inclusive",
     "if (lo[i - 1] < d && d <= hi[i - 1])", "if (lo[i - 1] <= d && d <= hi[i - 1])"),
    ("lists: hi bound exclusive",
     "if (lo[i - 1] < d && d <= hi[i - 1])", "if (lo[i - 1] < d && d < hi[i - 1])"),
    ("lists: no reset after a completion",
     "                count++;\n                for (int k = 0; k < N; k++) tl_clear(&s[k]);\n",
     "                count++;\n"),
    ("pruned: lo bound inclusive",
     "tt - P->v[P->head] > lo[i - 1]", "tt - P->v[P->head] >= lo[i - 1]"),
    ("pruned: entries dropped at exactly hi",
     "while (P->head < P->len && tt - P->v[P->head] > hi[i - 1]) P->head++;",
     "while (P->head < P->len && tt - P->v[P->head] >= hi[i - 1]) P->head++;"),
    # (In the exact machine the node order cannot change a count: an event is never
    # matched against its own time, since lo < delay is strict.  In the relaxed
    # machine, where zero delays are admitted, it can.)
    ("relaxed: nodes visited first to last",
     "                        const uint32_t *hi, uint8_t ty, uint32_t tt)\n{\n"
     "    for (int i = N - 1; i >= 0; i--) {",
     "                        const uint32_t *hi, uint8_t ty, uint32_t tt)\n{\n"
     "    for (int i = 0; i < N; i++) {"),
    ("relaxed: hi bound exclusive",
     "tt - s[i - 1] <= hi[i - 1]", "tt - s[i - 1] < hi[i - 1]"),
    ("relaxed: no reset after a completion",
     "            memset(set, 0, (size_t)N);\n", ""),
    ("relaxed: zero delays refused",
     "if (!(set[i - 1] && tt - s[i - 1] <= hi[i - 1])) continue;",
     "if (!(set[i - 1] && tt - s[i - 1] <= hi[i - 1] && tt != s[i - 1])) continue;"),
    ("mapconcat: window without the first edge",
     "for (int k = 0; k + 1 < N; k++) W += hi[k];", "for (int k = 1; k + 1 < N; k++) W += hi[k];"),
    ("printed mapconcat: machines do not start back by the summed hi",
     "            if (k > 0) back += hi[k - 1];\n", ""),
    ("printed mapconcat: cross-over window closed",
     "if (phase2 && tj >= tau[p + 1] + W) break;", "if (phase2 && tj > tau[p + 1] + W) break;"),
    ("mapconcat: class restarts at its own event",
     "int64_t from = c == ORC_NONE ? w : c + 1;", "int64_t from = c == ORC_NONE ? w : c;"),
]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_oracle_mistake(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {name}"
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(c)])
    env = dict(os.environ, FEM_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                        "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 1, f"the pins did not catch: {name}\n{r.stdout[-1500:]}"
