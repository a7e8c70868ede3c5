"""Planted mistakes: each test compiles a copy of the oracle with one plausible
error (a transposed index map, a dropped sign, a missing sqrt(m) scale, a wrong
tie rule, a transposed operand) and checks that the pins fail on it.  This is
the evidence that the pins constrain every part of the oracle's arithmetic; the
mutants exist only in a temporary directory, on the CPU."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = [
    # (name, original text, mistaken text, pin file that must fail)
    ("vec order of the HCS bins reversed", "stride *= mdims[k];", "stride *= mdims[N - 1 - k];",
     "test_oracle_projection.py"),
    ("reshape index map reversed", "int32_t ik = (int32_t)(r % dims[k]);",
     "int32_t ik = (int32_t)(r % dims[N - 1 - k]);", "test_oracle_projection.py"),
    ("count-sketch sign dropped", "y[h[i]] = y[h[i]] + (double)s[i] * x[i];",
     "y[h[i]] = y[h[i]] + x[i];", "test_oracle_projection.py"),
    ("sqrt(m) scale of Definitions 12/19 dropped", "? sqrt((double)m) : 1.0;", "? 1.0 : 1.0;",
     "test_oracle_projection.py"),
    ("SRP tie rule (zero gives 1)", "return y > 0.0 ? 1 : 0;", "return y >= 0.0 ? 1 : 0;",
     "test_oracle_discretize.py"),
    ("dense projection operand transposed",
     "acc = acc + x[j] * (double)G[(int64_t)j * ldg + col0 + l];",
     "acc = acc + x[j] * (double)G[(int64_t)l * ldg + col0 + j];", "test_oracle_projection.py"),
    ("floor replaced by truncation", "double f = floor(t3);", "double f = trunc(t3);",
     "test_oracle_discretize.py"),
    ("bucket ids not ordered inside a bucket", "return p->id < q->id ? -1 : (p->id > q->id ? 1 : 0);",
     "return p->id > q->id ? -1 : (p->id < q->id ? 1 : 0);", "test_oracle_index.py"),
    ("key folds swapped (ka and kb)", "return ((uint64_t)a << 32) | (uint64_t)b;",
     "return ((uint64_t)b << 32) | (uint64_t)a;", "test_oracle_key.py"),
    ("key fold without the mod 2^32 reduction", "uint32_t a = 0, b = 0;", "uint64_t a = 0, b = 0;",
     "test_oracle_key.py"),
    ("codes folded as 16-bit values", "a += (uint32_t)codes[l] * ka[l];",
     "a += (uint32_t)(uint16_t)codes[l] * ka[l];", "test_oracle_key.py"),
    ("key multiplier drawn from the low word", "ka[t * m + l] = (uint32_t)(r >> 32) | 1u;",
     "ka[t * m + l] = (uint32_t)r | 1u;", "test_oracle_key.py"),
    ("CSSRP-L bins of a column not distinct", "if (seen) continue;", "if (seen && 0) continue;",
     "test_oracle_csl.py"),
    ("CSSRP-L sign dropped", "y[h[e]] = y[h[e]] + (double)s[e] * x[i];", "y[h[e]] = y[h[e]] + x[i];",
     "test_oracle_csl.py"),
]


@pytest.mark.parametrize("name,orig,mutant,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, orig, mutant, pin):
    src = open(oracle._SRC).read()
    assert src.count(orig) >= 1, name  # every occurrence is mutated
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(orig, mutant))
    so = oracle.compile_to(str(mpath), str(tmp_path / "libmutant.so"))
    env = dict(os.environ, LSH_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu",
                        os.path.join(ROOT, "tests", pin)], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins in {pin} did not catch: {name}\n{r.stdout[-2000:]}"
