"""Planted-mistake checks: the oracle's pins must catch plausible errors.

Each mutant is a one-line edit of a copy of oracle/svdvals.c (a dropped term,
a wrong sign, an off-by-one index, a transposed operand).  The edited copy is
compiled on the CPU and run through a compact set of the same pins used in
test_oracle_pins.py; every mutant must fail at least one of them.  The real
oracle is never modified.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2608_21227_gb300 import inputs

EPS = np.finfo(np.float64).eps

MUTANTS = {
    # Householder: wrong tau normalisation
    "tau_over_alpha": ("return (b - alpha) / b;", "return (b - alpha) / alpha;"),
    # Householder: vector scaled by the wrong denominator
    "scale_sign": ("double scale = 1.0 / (alpha - b);", "double scale = 1.0 / (alpha + b);"),
    # left reflector misses its implicit unit entry
    "left_drop_head": ("double s = col[0];", "double s = 0.0;"),
    # right reflector applied to one row too few
    "right_rows_off_by_one": ("int r0 = j + 1, nr = m - r0;", "int r0 = j + 1, nr = m - r0 - 1;"),
    # right reflector skips the unit entry column
    "right_unit_col": ("double vc = (c == j + 1) ? 1.0 : vrow[IDX(0, c, lda)];",
                       "double vc = (c == j + 1) ? 0.0 : vrow[IDX(0, c, lda)];"),
    # last superdiagonal taken from the wrong entry
    "last_e_transposed": ("e[j] = A[IDX(j, j + 1, lda)];\n            continue;",
                          "e[j] = A[IDX(j + 1, j, lda)];\n            continue;"),
    # GK step: wrong sign in the left-rotation update of e
    "gk_e_sign": ("e[k] = c * ek + s * d[k + 1];", "e[k] = c * ek - s * d[k + 1];"),
    # GK step: the bulge carried to the next column is dropped
    "gk_drop_bulge": ("z = s * e[k + 1]; /* fill at (k, k+2) */", "z = 0.0 * e[k + 1];"),
    # norm: a dropped square in the sum of squares.  (A wrong *shift* is not a
    # mutant that changes results: every shift keeps the QR step orthogonal and
    # only changes how fast it converges.)
    "norm_no_square": ("        s += v * v;\n    }\n    if (s < DBL_MAX", "        s += fabs(v);\n    }\n    if (s < DBL_MAX"),
    # zero-diagonal chase: the fill is not propagated
    "chase_no_fill": ("x = -s * e[j];", "x = 0.0;"),
    # splitting test far too loose (drops real couplings)
    "split_loose": ("if (fabs(e[i]) <= eps * (fabs(d[i]) + fabs(d[i + 1]))) e[i] = 0.0;",
                    "if (fabs(e[i]) <= 1e-3 * (fabs(d[i]) + fabs(d[i + 1]))) e[i] = 0.0;"),
    # transpose decision inverted for wide matrices
    "no_transpose": ("int tr = m < n;", "int tr = 0;"),
}


def run_pins(lib):
    """Return the list of pin names that fail for the given library."""
    fails = []

    def rel(got, ref):
        return float(np.max(np.abs(np.asarray(got) - ref)) / max(ref[0], 1e-300))

    try:
        # closed form 2x2
        g = np.random.default_rng(101)
        for _ in range(30):
            a, b, c, d = g.standard_normal(4)
            s = a * a + b * b + c * c + d * d
            det = abs(a * d - b * c)
            s1 = np.sqrt((s + np.sqrt(max(s * s - 4 * det * det, 0))) / 2)
            ref = np.array([s1, det / s1])
            if rel(oracle.svdvals(np.array([[a, b], [c, d]]), lib=lib), ref) > 8 * EPS:
                fails.append("2x2")
                break
        # prescribed sigma, square and tall and wide
        for (m, n) in [(40, 40), (60, 35), (35, 60)]:
            sig = inputs.geometric_sigma(min(m, n), 1e6)
            A = inputs.prescribed(m, n, sig, seed=102 + m)
            if rel(oracle.svdvals(A, lib=lib), sig) > 1e-13 * max(m, n):
                fails.append(f"prescribed{m}x{n}")
        # Toeplitz bidiagonal closed form
        n = 30
        k = np.arange(1, n + 1)
        if rel(oracle.bdsvd(np.ones(n), np.ones(n - 1), lib=lib), 2 * np.cos(k * np.pi / (2 * n + 1))) > 8 * n * EPS:
            fails.append("toeplitz")
        # zero-diagonal bidiagonal against LAPACK
        g = np.random.default_rng(103)
        d = g.standard_normal(10)
        e = g.standard_normal(9)
        d[[3, 9]] = 0.0
        B = oracle.bidiagonal_dense(d, e)
        if rel(oracle.bdsvd(d, e, lib=lib), np.linalg.svd(B, compute_uv=False)) > 50 * EPS:
            fails.append("zero-diag")
        # Frobenius invariant
        A = inputs.gaussian(50, 30, 104)
        s = oracle.svdvals(A, lib=lib)
        if abs(np.sum(s * s) - np.sum(A * A)) > 1e-13 * 50 * np.sum(A * A):
            fails.append("frobenius")
    except (RuntimeError, ValueError, FloatingPointError) as ex:  # non-convergence counts as caught
        fails.append(f"error:{ex}")
    return fails


def test_real_oracle_passes_compact_pins():
    assert run_pins(oracle.load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = oracle.compile_variant(src.replace(old, new), os.path.join(tmp_path, f"mut_{name}.so"))
    lib = oracle.load(path)
    assert run_pins(lib), f"mutant {name} passed every pin"
