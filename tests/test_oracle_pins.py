"""Pins for the FP64 oracle (CPU only).

The oracle computes the singular values of a dense matrix (paper Section
5.1.1: orthogonal reduction keeps the singular values intact).  Each test here
checks it against something other than itself: closed forms, invariants,
special cases that reduce to a textbook result, a LAPACK library routine run
only as a cross-check, and a second independent algorithm (one-sided Jacobi).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2608_21227_gb300 import inputs

EPS = np.finfo(np.float64).eps


def err_rel(got, ref):
    """max_i |got_i - ref_i| / ref_1 (absolute singular-value error relative to sigma_max)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape
    if ref.size == 0:
        return 0.0
    scale = ref[0] if ref[0] > 0 else 1.0
    return float(np.max(np.abs(got - ref)) / scale)


# ---------------------------------------------------------------- closed forms

def closed_form_2x2(a, b, c, d):
    # sigma_{1,2}^2 = (S +- sqrt(S^2 - 4 D^2)) / 2, S = a^2+b^2+c^2+d^2, D = |ad - bc|;
    # evaluated on the matrix divided by its largest entry to avoid overflow.
    t = max(abs(a), abs(b), abs(c), abs(d))
    if t == 0:
        return np.zeros(2)
    a, b, c, d = a / t, b / t, c / t, d / t
    s = a * a + b * b + c * c + d * d
    det = abs(a * d - b * c)
    disc = math.sqrt(max(s * s - 4 * det * det, 0.0))
    s1 = math.sqrt((s + disc) / 2)
    # the smaller root in a cancellation-free form: s1 * s2 = |det|
    s2 = det / s1
    return t * np.array([s1, s2])


def test_2x2_closed_form():
    g = np.random.default_rng(11)
    cases = [g.standard_normal(4) for _ in range(200)]
    cases += [np.array(v, dtype=float) for v in
              ([0, 0, 0, 0], [1, 2, 2, 4], [3, 0, 0, -5], [0, 1, 0, 0], [0, 0, 1, 0],
               [1e-300, 0, 0, 1e300], [1, 1, 1, 1 + 1e-12])]
    for v in cases:
        a, b, c, d = v
        A = np.array([[a, b], [c, d]])
        ref = closed_form_2x2(a, b, c, d)
        got = oracle.svdvals(A)
        assert err_rel(got, ref) <= 8 * EPS, (v, got, ref)


def test_diagonal_rectangular():
    g = np.random.default_rng(12)
    for (m, n) in [(1, 1), (5, 5), (7, 4), (4, 7), (40, 33)]:
        p = min(m, n)
        dg = g.standard_normal(p) * 10.0 ** g.integers(-3, 4, size=p)
        dg[p // 2] = 0.0
        A = np.zeros((m, n))
        A[np.arange(p), np.arange(p)] = dg
        ref = np.sort(np.abs(dg))[::-1]
        got = oracle.svdvals(A)
        assert err_rel(got, ref) <= 4 * EPS


@pytest.mark.parametrize("m,n", [(1, 1), (2, 2), (64, 64), (200, 200), (150, 60), (60, 150)])
def test_orthonormal_all_ones(m, n):
    g = np.random.default_rng(13 + m + n)
    if m >= n:
        A = inputs.haar(m, n, g)
    else:
        A = inputs.haar(n, m, g).T
    got = oracle.svdvals(A)
    assert np.max(np.abs(got - 1.0)) <= 20 * max(m, n) * EPS


@pytest.mark.parametrize("m,n", [(30, 30), (80, 45), (45, 80), (1, 9)])
def test_rank_one(m, n):
    g = np.random.default_rng(14)
    u = g.standard_normal(m)
    v = g.standard_normal(n)
    A = np.outer(u, v)
    got = oracle.svdvals(A)
    s1 = np.linalg.norm(u) * np.linalg.norm(v)
    assert abs(got[0] - s1) <= 10 * max(m, n) * EPS * s1
    assert np.all(np.abs(got[1:]) <= 10 * max(m, n) * EPS * s1)


@pytest.mark.parametrize("m,n,kappa", [(64, 64, 1e6), (120, 80, 1e12), (80, 120, 1e3),
                                       (100, 100, 1.0), (257, 256, 1e8)])
def test_prescribed_sigma(m, n, kappa):
    p = min(m, n)
    sigma = inputs.geometric_sigma(p, kappa)
    A = inputs.prescribed(m, n, sigma, seed=15 + m)
    got = oracle.svdvals(A)
    N = max(m, n)
    assert err_rel(got, sigma) <= 1e-13 * N


def test_frobenius_invariant():
    for seed, (m, n) in enumerate([(50, 50), (97, 31), (31, 97), (300, 280)]):
        A = inputs.gaussian(m, n, 16 + seed)
        s = oracle.svdvals(A)
        fro2 = float(np.sum(A * A))
        assert abs(np.sum(s * s) - fro2) <= 1e-13 * max(m, n) * fro2


# ---------------------------------------------------------------- bidiagonal solver

@pytest.mark.parametrize("n", [1, 2, 3, 10, 101, 400])
def test_bdsvd_toeplitz_closed_form(n):
    # Golub-Kahan form of B(d=1, e=1) is the 2n x 2n tridiagonal Toeplitz matrix
    # with zero diagonal and unit off-diagonals: eigenvalues 2 cos(k pi / (2n+1)).
    got = oracle.bdsvd(np.ones(n), np.ones(n - 1))
    k = np.arange(1, n + 1)
    ref = 2 * np.cos(k * np.pi / (2 * n + 1))
    assert err_rel(got, ref) <= 8 * n * EPS


def test_bdsvd_scaled_toeplitz():
    # d_i = a, e_i = b: TGK is Toeplitz with alternating a, b off-diagonals; for
    # a = b it reduces to the case above scaled by a.
    n = 57
    for a in (1e-200, 3.5, 1e200):
        got = oracle.bdsvd(np.full(n, a), np.full(n - 1, a))
        k = np.arange(1, n + 1)
        ref = 2 * a * np.cos(k * np.pi / (2 * n + 1))
        assert err_rel(got, ref) <= 8 * n * EPS


def test_bdsvd_diagonal():
    g = np.random.default_rng(17)
    d = g.standard_normal(40)
    got = oracle.bdsvd(d, np.zeros(39))
    assert err_rel(got, np.sort(np.abs(d))[::-1]) == 0.0


@pytest.mark.parametrize("zeros", [[0], [3], [9], [0, 4, 9], [5, 6]])
def test_bdsvd_zero_diagonal(zeros):
    # zero diagonal entries exercise the zero-shift chase (GvL Sec. 8.6.2);
    # reference: the dense bidiagonal through the Jacobi oracle and LAPACK.
    g = np.random.default_rng(18)
    d = g.standard_normal(10)
    e = g.standard_normal(9)
    d[zeros] = 0.0
    got = oracle.bdsvd(d, e)
    B = oracle.bidiagonal_dense(d, e)
    ref = np.linalg.svd(B, compute_uv=False)
    assert err_rel(got, ref) <= 50 * EPS
    assert err_rel(got, oracle.jacobi_svdvals(B)) <= 50 * EPS


def test_bdsvd_graded():
    # strongly graded bidiagonal, values spanning 1e-12..1
    n = 60
    d = 10.0 ** (-12 * np.arange(n) / (n - 1))
    e = 0.5 * d[:-1]
    got = oracle.bdsvd(d, e)
    ref = np.linalg.svd(oracle.bidiagonal_dense(d, e), compute_uv=False)
    assert err_rel(got, ref) <= 50 * n * EPS


# ---------------------------------------------------------------- bidiagonalisation

@pytest.mark.parametrize("m,n", [(1, 1), (2, 2), (3, 2), (33, 17), (64, 64), (129, 100)])
def test_bidiag_structure_and_values(m, n):
    A = inputs.gaussian(m, n, 19 + m)
    d, e = oracle.bidiag(A)
    # Frobenius norm is preserved by the orthogonal reduction
    fro2 = float(np.sum(A * A))
    assert abs(np.sum(d * d) + np.sum(e * e) - fro2) <= 1e-13 * m * fro2
    # the bidiagonal has the singular values of A (LAPACK cross-check)
    ref = np.linalg.svd(A, compute_uv=False)
    got = np.linalg.svd(oracle.bidiagonal_dense(d, e), compute_uv=False)
    assert err_rel(got, ref) <= 1e-13 * m


# ---------------------------------------------------------------- metamorphic

def test_metamorphic():
    g = np.random.default_rng(20)
    A = inputs.gaussian(70, 50, 21)
    s = oracle.svdvals(A)
    N = 70
    assert err_rel(oracle.svdvals(-3.25 * A), 3.25 * s) <= 1e-13 * N
    assert err_rel(oracle.svdvals(A.T), s) <= 1e-13 * N
    Q1 = inputs.haar(70, 70, g)
    Q2 = inputs.haar(50, 50, g)
    assert err_rel(oracle.svdvals(Q1 @ A @ Q2), s) <= 1e-13 * N
    B = inputs.gaussian(20, 30, 22)
    sb = oracle.svdvals(B)
    C = np.zeros((90, 80))
    C[:70, :50] = A
    C[70:, 50:] = B
    # 80 values: the 50 + 20 block values plus 10 exact zeros (rank <= 70)
    ref = np.sort(np.concatenate([s, sb, np.zeros(10)]))[::-1]
    assert err_rel(oracle.svdvals(C), ref) <= 1e-13 * 90


# ---------------------------------------------------------------- cross-checks

@pytest.mark.parametrize("m,n", [(1, 5), (5, 1), (17, 17), (100, 37), (37, 100), (256, 256), (500, 300)])
def test_lapack_crosscheck(m, n):
    A = inputs.uniform(m, n, 23 + m + n)
    got = oracle.svdvals(A)
    ref = np.linalg.svd(A, compute_uv=False)
    assert err_rel(got, ref) <= 1e-13 * max(m, n)


@pytest.mark.parametrize("m,n", [(8, 8), (40, 25), (25, 40), (64, 64)])
def test_jacobi_crosscheck(m, n):
    A = inputs.gaussian(m, n, 24 + m)
    assert err_rel(oracle.svdvals(A), oracle.jacobi_svdvals(A)) <= 1e-13 * max(m, n)


def test_jacobi_pins():
    # the second oracle is pinned by the same closed forms
    g = np.random.default_rng(25)
    for _ in range(20):
        v = g.standard_normal(4)
        A = v.reshape(2, 2)
        assert err_rel(oracle.jacobi_svdvals(A), closed_form_2x2(*v)) <= 8 * EPS
    Q = inputs.haar(30, 30, g)
    assert np.max(np.abs(oracle.jacobi_svdvals(Q) - 1)) <= 100 * EPS


def test_empty_and_thread_counts():
    assert oracle.svdvals(np.zeros((0, 4))).shape == (0,)
    assert oracle.svdvals(np.zeros((4, 0))).shape == (0,)
    A = inputs.gaussian(90, 60, 26)
    s1 = oracle.svdvals(A, nthreads=1)
    s4 = oracle.svdvals(A, nthreads=4)
    assert err_rel(s1, s4) <= 1e-14
