"""Pins for the oracle's dense kernels (oracle/liboracle.c).

* Householder QR against LAPACK (numpy.linalg.qr): same R up to row signs,
  orthogonal Q, Q R = A.
* Triangular solves against SciPy's solve_triangular.
* The QR least-squares solve against an extended-precision (mpmath, 60
  digits) normal-equations solve on tiny inputs, and against LAPACK lstsq.
* Compensated residual against an exact rational evaluation.
* The extreme singular values of R on constructed spectra and the 2 x 2
  closed forms (determinant, Frobenius norm).
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import lsq_oracle as O
from lsq_problems import problem_svd

mpmath = pytest.importorskip("mpmath")


@pytest.mark.parametrize("m,n", [(50, 7), (300, 40), (64, 64), (1000, 3)])
def test_householder_matches_lapack(m, n):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)) * np.logspace(0, -6, n)
    R, V = O.householder_qr(A)
    _, R_ref = np.linalg.qr(A)
    s = np.sign(np.diag(R)) * np.sign(np.diag(R_ref))
    assert np.allclose(R, s[:, None] * R_ref, rtol=0, atol=1e-13 * np.abs(R_ref).max())
    assert np.allclose(np.tril(R, -1), 0.0)
    # Q^T A = [R; 0] with Q^T applied column by column
    QtA = np.stack([O.apply_qt(V, A[:, j]) for j in range(n)], axis=1)
    assert np.allclose(QtA[:n], R, atol=1e-13 * np.abs(A).max())
    assert np.allclose(QtA[n:], 0.0, atol=1e-13 * np.abs(A).max())
    # Q^T is orthogonal: it preserves norms
    y = rng.standard_normal(m)
    assert abs(np.linalg.norm(O.apply_qt(V, y)) - np.linalg.norm(y)) < 1e-13 * np.linalg.norm(y)


def test_householder_zero_column():
    A = np.zeros((6, 3))
    A[:, 0] = 1.0
    A[:, 2] = np.arange(6.0)
    R, _ = O.householder_qr(A)
    assert abs(abs(R[0, 0]) - np.sqrt(6.0)) < 1e-14
    assert np.isfinite(R).all()


@pytest.mark.parametrize("n", [1, 5, 60])
def test_triangular_solves(n):
    rng = np.random.default_rng(n)
    R = np.triu(rng.standard_normal((n, n))) + 3 * np.eye(n)
    y = rng.standard_normal(n)
    assert np.allclose(O.backsub(R, y), sl.solve_triangular(R, y), rtol=1e-13, atol=1e-14)
    assert np.allclose(O.backsub_t(R, y), sl.solve_triangular(R, y, trans="T"), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_qr_solve_extended_precision(seed):
    rng = np.random.default_rng(seed)
    m, n = 9, 3
    A = rng.standard_normal((m, n))
    A[:, 2] = A[:, 0] + 1e-5 * A[:, 2]            # moderately ill-conditioned
    b = rng.standard_normal(m)
    x = O.qr_solve(A, b)
    mpmath.mp.dps = 60
    Am = mpmath.matrix(A.tolist())
    bm = mpmath.matrix(b.tolist())
    xm = mpmath.lu_solve(Am.T * Am, Am.T * bm)   # exact-ish normal equations
    x_ref = np.array([float(v) for v in xm])
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 50 * kappa ** 2 * 2.0 ** -53 * 10


def test_qr_solve_matches_lstsq_constructed():
    P = problem_svd(2000, 30, 1e6, 1e-4, seed=8)
    x = O.qr_solve(P["A"], P["b"])
    x_l = np.linalg.lstsq(P["A"], P["b"], rcond=None)[0]
    wb = O.wedin_bound(1e6, 1.0, P["x_true"], 1e-4)
    assert O.forward_error(x, P["x_true"]) < wb
    assert O.forward_error(x, x_l) < 2 * wb


def test_residual_dot2_exact():
    rng = np.random.default_rng(5)
    m, n = 40, 6
    A = rng.standard_normal((m, n))
    x = rng.standard_normal(n)
    b = A @ x + 1e-12 * rng.standard_normal(m)     # heavy cancellation in b - A x
    r_hi, r_lo, g = O.residual_dot2(A, b, x)
    F = [[Fraction(v) for v in row] for row in A]
    fx = [Fraction(v) for v in x]
    r_ex = [Fraction(b[i]) - sum(F[i][j] * fx[j] for j in range(n)) for i in range(m)]
    g_ex = [sum(F[i][j] * r_ex[i] for i in range(m)) for j in range(n)]
    r_ex_f = np.array([float(v) for v in r_ex])
    g_ex_f = np.array([float(v) for v in g_ex])
    assert np.allclose(r_hi, r_ex_f, rtol=4e-16, atol=0)
    assert np.allclose(g, g_ex_f, rtol=1e-14, atol=1e-16 * np.abs(g_ex_f).max())


def test_wedin_bound_hand_values():
    """Fact 2.4's forward-error bound, relative to ||x||, at points evaluated
    by hand: 2.23 kappa (||x|| + kappa ||r|| / ||A||) u / ||x||."""
    u = 2.0 ** -53
    x = np.array([3.0, 4.0])                      # ||x|| = 5
    # kappa 1e6, ||A|| 2, ||r|| 1e-3: 2.23e6 (5 + 500) / 5 = 2.2523e8
    assert abs(O.wedin_bound(1e6, 2.0, x, 1e-3) / (2.2523e8 * u) - 1) < 1e-12
    # kappa 1e8, ||A|| 1, ||r|| 1e-2: 2.23e8 (5 + 1e6) / 5 = 4.46002230e13
    assert abs(O.wedin_bound(1e8, 1.0, x, 1e-2) / (4.4600223e13 * u) - 1) < 1e-12
    # zero residual: 2.23 kappa
    assert abs(O.wedin_bound(1e10, 1.0, x, 0.0) / (2.23e10 * u) - 1) < 1e-12
    # eps other than u enters linearly
    assert abs(O.wedin_bound(1e3, 1.0, x, 0.0, u=1e-8) / (2.23e-5) - 1) < 1e-12


def _exact_ls_orthogonal_columns(cols, b):
    """Exact least-squares solution when the columns are mutually
    orthogonal: x_j = a_j^T b / ||a_j||^2 (rational arithmetic)."""
    return [sum(a * bi for a, bi in zip(c, b)) / sum(a * a for a in c) for c in cols]


@pytest.mark.parametrize("term", ["kappa_x", "kappa2_r"])
def test_wedin_bound_is_attained(term):
    """Fact 2.4 is tight to its constant: on A = [e1, delta e2] (3 x 2,
    ||A|| = 1, kappa = 1/delta) a perturbation with ||Delta A|| = eps moves x
    by eps kappa ||x|| (zero residual; Delta A scales the second column) or
    by eps kappa^2 ||r|| (residual r = rho e3; Delta A tilts the second column
    towards r).  The exact perturbed solutions (rational arithmetic) must lie
    below the bound and above 0.4 of it (the first-order error is 1 / 2.23 of
    the bound), so a dropped term or a wrong constant fails."""
    F = Fraction
    delta, eps = F(1, 10 ** 4), F(1, 10 ** 12)
    kappa = 1 / delta
    if term == "kappa_x":
        x = [F(0), F(1)]
        rho = F(0)
        cols_p = [[F(1), F(0), F(0)], [F(0), delta + eps, F(0)]]
    else:
        x = [F(1), F(1)]
        rho = F(1)
        cols_p = [[F(1), F(0), F(0)], [F(0), delta, eps]]
    b = [x[0], delta * x[1], rho]                 # A x + rho e3, r = rho e3 orthogonal to range(A)
    xp = _exact_ls_orthogonal_columns(cols_p, b)
    err = math.sqrt(float(sum((p - q) ** 2 for p, q in zip(xp, x))))
    nx = math.sqrt(float(sum(v * v for v in x)))
    bound = O.wedin_bound(float(kappa), 1.0, np.array([float(v) for v in x]), float(rho),
                          u=float(eps)) * nx
    assert err <= bound, (err, bound)
    assert err >= 0.4 * bound, (err, bound)


def test_qr_solve_lapack_matches_plain_loops():
    """The LAPACK-backed solve (for the large bench problems) against the
    oracle's plain Householder loops: R equal up to row signs, x within the
    Wedin bound of the known solution and of the plain solve."""
    P = problem_svd(3000, 40, 1e8, 1e-4, seed=12)
    x, R = O.qr_solve(P["A"], P["b"], return_R=True)
    xl, Rl = O.qr_solve_lapack(P["A"], P["b"], return_R=True)
    s = np.sign(np.diag(R)) * np.sign(np.diag(Rl))
    assert np.allclose(Rl * s[:, None], R, rtol=0, atol=1e-12 * np.abs(R).max())
    wb = O.wedin_bound(1e8, 1.0, P["x_true"], 1e-4)
    assert O.forward_error(xl, P["x_true"]) < wb
    assert O.forward_error(xl, x) < 2 * wb
    # the KW estimate is the same whichever R it is given
    be = O.kw_relative(P["A"], P["b"], xl, R_A=R)
    bel = O.kw_relative(P["A"], P["b"], xl, R_A=Rl)
    assert abs(be - bel) <= 1e-6 * be


@pytest.mark.parametrize("n,kappa", [(6, 1e3), (40, 1e10)])
def test_sigma_extremes_constructed(n, kappa):
    """sigma_extremes (the extreme singular values of R, used for the condition
    estimates) on R factors whose singular values are fixed by construction:
    orthogonal transformations keep them, so the R of U diag(s) V^T (U, V from
    QRs of Gaussians) has singular values s."""
    rng = np.random.default_rng(n)
    s = np.logspace(0, -math.log10(kappa), n) * 3.0
    U, _ = np.linalg.qr(rng.standard_normal((5 * n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    R, _ = O.householder_qr((U * s) @ V.T)
    smax, smin = O.sigma_extremes(R)
    assert abs(smax - s[0]) <= 1e-13 * s[0]
    # the smallest one to the accuracy the QR leaves it: ~u sigma_max
    assert abs(smin - s[-1]) <= 1e-14 * s[0] * n


def test_sigma_extremes_two_by_two():
    """For R = [[a, b], [0, c]]: sigma_max sigma_min = |a c| (the determinant) and
    sigma_max^2 + sigma_min^2 = a^2 + b^2 + c^2 (the Frobenius norm)."""
    for a, b, c in [(3.0, 4.0, 2.0), (1.0, 0.0, 1e-8), (-2.0, 7.0, 0.5)]:
        smax, smin = O.sigma_extremes(np.array([[a, b], [0.0, c]]))
        assert smax >= smin > 0.0
        assert abs(smax * smin - abs(a * c)) <= 1e-14 * smax * smax
        assert abs(smax ** 2 + smin ** 2 - (a * a + b * b + c * c)) <= 1e-14 * (a * a + b * b + c * c)
