"""The pins are not a restatement of the oracle: each plausible mistake planted in a copy of
the oracle's source (a dropped or wrong term, a sign, an index, a comparison) makes at least
one pin fail.  CPU only: every mutant is compiled with gcc into a temporary directory and
the pin suite runs against it in a subprocess (RBFFD_ORACLE_TEST_LIB)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rbffd_oracle.c")

# (what, text in the oracle, replacement): the first occurrence is replaced
MUTANTS = [
    ("Laplacian coefficient of r^m", "v = (double)(m * (m + d - 2)) * odd_power(r, r2, m - 2);",
     "v = (double)(m * (m + d - 1)) * odd_power(r, r2, m - 2);"),
    ("power in the right-hand side", "v = (double)(m * (m + d - 2)) * odd_power(r, r2, m - 2);",
     "v = (double)(m * (m + d - 2)) * odd_power(r, r2, m);"),
    ("sign in the forward substitution",
     "for (int j = 0; j < i; ++j) s = s - A[i * K + j] * b[j];",
     "for (int j = 0; j < i; ++j) s = s + A[i * K + j] * b[j];"),
    ("polynomial block not the transpose", "A[(n + l) * K + i] = v;",
     "A[(n + l) * K + i] = mono(xi + i * d, alpha + ((l + 1) % M) * d, d);"),
    ("weights not scaled back", "W[j * q + e] = (op == ORA_OP_LAPLACIAN) ? col[j] / rho2",
     "W[j * q + e] = (op == ORA_OP_LAPLACIAN) ? col[j] / rho"),
    ("open retention ball", "if (d2[k * n + t] <= r2) len = t + 1;",
     "if (d2[k * n + t] < r2) len = t + 1;"),
    ("kNN ties to the higher index", "(s == bd[pos - 1] && j < bi[pos - 1])",
     "(s == bd[pos - 1] && j > bi[pos - 1])"),
    ("covered nodes recomputed", "if (!covered[I[t]] && !(bc && bc[I[t]])) cols[q++] = t;",
     "if (!(bc && bc[I[t]])) cols[q++] = t;"),
    ("Lebesgue test threshold", "pass = lam[e] <= lam[e_ref];",
     "pass = lam[e] < 0.95 * lam[e_ref];"),
    ("centroid reference ignored", "pass = lam[e] <= lam[e_ref];",
     "pass = lam[e] <= lam[0];"),
    ("centroid divided by n - 1", "c[a] = s / (double)n;", "c[a] = s / (double)(n - 1);"),
    ("centroid sum skips the center", "for (int t = 0; t < n; ++t) s = s + X[(int64_t)I[t] * d + a];",
     "for (int t = 1; t < n; ++t) s = s + X[(int64_t)I[t] * d + a];"),
]


def _run_pins(tmp_path, src):
    """Compile `src` as the oracle and run the pin suite against it; returns the result."""
    (tmp_path / "rbffd_oracle.c").write_text(src)
    (tmp_path / "rbffd_oracle.h").write_text(open(os.path.join(ROOT, "oracle",
                                                               "rbffd_oracle.h")).read())
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", str(lib), str(tmp_path / "rbffd_oracle.c"),
                           "-lm"])
    env = dict(os.environ, RBFFD_ORACLE_TEST_LIB=str(lib))
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_an_unchanged_copy_passes_every_pin(tmp_path):
    """Control: the same route with the oracle's own source passes."""
    r = _run_pins(tmp_path, open(SRC).read())
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_every_planted_mistake_fails_a_pin(what, old, new, tmp_path):
    src = open(SRC).read()
    assert old in src, what
    r = _run_pins(tmp_path, src.replace(old, new, 1))
    assert r.returncode != 0, f"no pin caught: {what}\n{r.stdout[-2000:]}"
