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

PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_backward.py",
        "tests/test_oracle_derived.py"]
DERIVED = ["tests/test_oracle_derived.py"]  # pins of the derived transforms alone

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
    ("d c / d lambda with the wrong sign", "REAL dc = (di2 - s2[k]) / (c + c);",
     "REAL dc = (s2[k] - di2) / (c + c);"),
    ("d c / d lambda without the factor 1/2", "REAL dc = (di2 - s2[k]) / (c + c);",
     "REAL dc = (di2 - s2[k]) / c;"),
    ("lambda term from the parent's adjoint", "*lt = *lt + g[xi] * dc;",
     "*lt = *lt + g[yi] * dc;"),
    ("v terms without the mask", "v_terms[i] = mask[i] * G[i];", "v_terms[i] = G[i];"),
    ("signed transform without the complement",
     "comp = (np.float32(1.0) - m).astype(np.float32)", "comp = m.copy()", "__init__.py"),
    ("signed transform with the terms swapped", "return (a - b).astype(np.float32)",
     "return (b - a).astype(np.float32)", "__init__.py"),
    ("GSF threshold difference with the wrong sign", "c = np.float32(td - te)",
     "c = np.float32(te - td)", "__init__.py", DERIVED),
    ("GSF erosion on the wrong side", "f_e = (s < -te).astype(np.float32)",
     "f_e = (s < te).astype(np.float32)", "__init__.py", DERIVED),
    ("GSF signed distance of the background",
     "        comp = (np.float32(1.0) - x).astype(np.float32)\n",
     "        comp = x.copy()\n", "__init__.py", DERIVED),
    ("GSF erosion in place of the dilation",
     "total = (signed_of_object(f_e) + signed_of_object(f_d))",
     "total = (signed_of_object(f_e) + signed_of_object(f_e))", "__init__.py", DERIVED),
]


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_planted_mistake(tmp_path, mutant):
    label, old, new = mutant[:3]
    fname = mutant[3] if len(mutant) > 3 else "gdt_core.inc"
    pins = mutant[4] if len(mutant) > 4 else PINS
    for d in ("oracle", "tests", "workloads"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")
    src = tmp_path / "oracle" / fname
    text = src.read_text()
    assert old in text, label
    src.write_text(text.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", *pins],
                       cwd=tmp_path, capture_output=True, text=True, timeout=900)
    assert r.returncode != 0, f"pins did not catch: {label}\n{r.stdout[-2000:]}"
