"""Pins of the oracle's complex path (the Prony experiment's complex
least-squares problems, solved through the real embedding): the embedding
against complex arithmetic, the Karlson-Walden estimate on the embedding
against the estimate evaluated directly in complex arithmetic through the
SVD of A (Sec. 4.1's display; App. A.1's SVD form), and the complex FOSSILS
/ SPIR answers against LAPACK's complex least-squares solver."""
import math

import numpy as np
import pytest

import oracle
from lsq_problems import problem_prony

u = 2.0 ** -53


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_real_embedding_products():
    """E x_r is A x (interleaved), E^T r_r is A^H r, ||E||_F = sqrt(2) ||A||_F,
    and the singular values of E are those of A, each twice."""
    rng = np.random.default_rng(5)
    A = _crandn(rng, 9, 4)
    x = _crandn(rng, 4)
    r = _crandn(rng, 9)
    E = oracle.real_embedding(A)
    assert E.shape == (18, 8)
    assert np.allclose(E @ oracle.as_real(x), oracle.as_real(A @ x), rtol=0, atol=1e-14)
    assert np.allclose(E.T @ oracle.as_real(r), oracle.as_real(A.conj().T @ r), rtol=0, atol=1e-14)
    assert math.isclose(np.linalg.norm(E), math.sqrt(2) * np.linalg.norm(A), rel_tol=1e-15)
    sA = np.linalg.svd(A, compute_uv=False)
    sE = np.linalg.svd(E, compute_uv=False)
    assert np.allclose(sE, np.repeat(sA, 2), rtol=1e-14)
    assert np.array_equal(oracle.as_complex(oracle.as_real(x)), x)


def _kw_complex_svd(A, b, x):
    """Sec. 4.1's estimate in complex arithmetic through A = U S V^H:
    theta / sqrt(1 + theta^2 ||x||^2) || (S^2 + lam)^{-1/2} S U^H r ||."""
    U, S, Vh = np.linalg.svd(A, full_matrices=False)
    theta = np.linalg.norm(A) / np.linalg.norm(b)
    r = b - A @ x
    nx = np.linalg.norm(x)
    lam = theta ** 2 * np.linalg.norm(r) ** 2 / (1 + theta ** 2 * nx ** 2)
    y = S * (U.conj().T @ r) / np.sqrt(S ** 2 + lam)
    return theta / math.sqrt(1 + theta ** 2 * nx ** 2) * np.linalg.norm(y) / np.linalg.norm(A)


@pytest.mark.parametrize("scale", [1e-3, 1e-7])
def test_kw_complex_matches_svd_form(scale):
    """At perturbed least-squares solutions (the estimate well above the
    rounding of its own evaluation) the embedding's estimate equals the
    complex SVD form to 1e-8 relative."""
    rng = np.random.default_rng(11)
    A = _crandn(rng, 300, 12) @ np.diag(10.0 ** rng.uniform(-3, 0, 12))
    b = _crandn(rng, 300)
    x = np.linalg.lstsq(A, b, rcond=None)[0]
    xp = x + scale * np.linalg.norm(x) * _crandn(rng, 12) / math.sqrt(24)
    got = oracle.kw_relative_complex(A, b, xp)
    ref = _kw_complex_svd(A, b, xp)
    assert abs(got - ref) <= 1e-8 * ref, (got, ref)


@pytest.mark.parametrize("method", ["fossils", "spir"])
def test_complex_prony_against_lapack(method):
    """A Prony-shaped complex problem (4000 x 20, condition ~1e6): the
    oracle's method on the real embedding is backward stable in the complex
    sense and agrees with LAPACK's complex least-squares solution to within
    the Wedin-type level kappa^2 u (the residual is not small)."""
    P = problem_prony(4000, 20, seed=1)
    A, b = P["A"], P["b"]
    x, res = oracle.solve_complex(method, A, b, seed=3)
    assert oracle.kw_relative_complex(A, b, x) <= 1e-14
    xl = np.linalg.lstsq(A, b, rcond=None)[0]
    kappa = np.linalg.cond(A)
    r = b - A @ xl
    bound = 2.23 * kappa * (1 + kappa * np.linalg.norm(r) / (np.linalg.norm(A, 2) * np.linalg.norm(xl))) * u
    assert np.linalg.norm(x - xl) / np.linalg.norm(xl) <= 10 * bound
    # the real method took the real embedding's step counts
    assert res["iters"][0] >= 1 and len(res["iters"]) == 2
