"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a private copy of the oracle's C source (a
dropped term, a wrong sign or index, a swapped operand), rebuilds that copy in
a temporary directory and runs the pin tests against it in a subprocess; the
pins must fail.  The real oracle is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = [
    ("drop the W term of |x-y|^2", "REAL s2 = (e0 * e0 + e1 * e1) + e2 * e2;",
     "REAL s2 = (e0 * e0 + e1 * e1);"),
    ("drop lambda on the intensity term", "REAL u = lambda * di2;", "REAL u = di2;"),
    ("drop the spatial term", "REAL c = SQRT(t[k] + u);", "REAL c = SQRT(u);"),
    ("previous line on the wrong side", "const int64_t ya = xa - s; ",
     "const int64_t ya = xa + s; "),
    ("in-line offset on the wrong axis", "delta[qa] = (REAL)dq;", "delta[qa] = (REAL)dp;"),
    ("skip the first updated line", "for (int64_t l = 1; l < L; ++l) {",
     "for (int64_t l = 2; l < L; ++l) {"),
    ("lambda instead of 1 - lambda", "REAL one_minus = (REAL)1 - lambda;",
     "REAL one_minus = lambda;"),
    ("parent ignores its children", "acc = acc + g[xi];", "acc = acc + 0 * g[xi];"),
    ("wrong sign of the parent's image term",
     "gi[ch * N + yi] = gi[ch * N + yi] - w * d;", "gi[ch * N + yi] = gi[ch * N + yi] + w * d;"),
    ("sum of differences instead of squares", "di2 = di2 + d * d;", "di2 = di2 + d;"),
]


@pytest.mark.parametrize("label,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_planted_mistake(tmp_path, label, old, new):
    for d in ("oracle", "tests", "workloads"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")
    src = tmp_path / "oracle" / "gdt_core.inc"
    text = src.read_text()
    assert old in text, label
    src.write_text(text.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q",
                        "tests/test_oracle_pins.py", "tests/test_oracle_backward.py"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=900)
    assert r.returncode != 0, f"pins did not catch: {label}\n{r.stdout[-2000:]}"
