"""Pins for the oracle's solvers (oracle/lsq_oracle.py).

* q0 (Theorem 7.1) at hand-evaluated points, including the floor of 11.
* Polyak heavy ball (Alg. 5) against the exact-arithmetic error bound
  4 sqrt(2) j eta^{j-2} ||c|| of the Polyak-with-noise lemma (Sec. 7.1), and
  the eta = 0 special case (identity preconditioned operator: exact after one
  update).
* CG against finite termination on a small SPD system.
* LSQR (the inner solver of LSQR-based SPIR) against CG's iterates on the
  same preconditioned problem (identical in exact arithmetic) and against
  LAPACK lstsq after convergence; LSQR-based SPIR on constructed problems.
* The sketched Karlson-Walden estimate (eq. (sketched-kw)) against the KW
  estimate when the "sketch" is A itself, against the Proposition's bounds
  for a sparse sign sketch, and Alg. 4's step-2 test built on it.
* FOSSILS / SPIR on constructed problems with known solution: backward error
  <= 1e-13 (Karlson-Walden, Sec. 4.1), forward error within 10x of the
  Householder QR solve, two refinement steps needed (Sec. 5.1), and the
  paper's printed numbers of Table 1 and Table 2 (tests/golden/).
* The Karlson-Walden estimate against its closed form in a known SVD basis
  (App. A.1, proof of Theorem 2.8, with theta kept general) and against the
  bound BE-hat <= BE <= ||Delta A||_F for an exactly solved perturbed problem.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import lsq_oracle as O
from lsq_problems import problem_svd

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
u = 2.0 ** -53


def test_q0_values():
    eta = math.sqrt(1 / 12)
    # 1 + 2 ln(1/(1e12 u)) / ln(1/(1.01 eta)) evaluated by hand: 15.776...
    assert abs(O.q0_count(1e12, eta) - 15.7762) < 1e-3
    assert abs(O.q0_count(1e10, eta) - 23.2493) < 1e-3
    assert O.q0_count(1e20, eta) == 11.0
    assert O.step2_updates(1e12, eta) == 15
    assert O.step2_updates(1e4, eta, max_inner=30) == 30


class _Op:
    def __init__(self, M):
        self.M = M

    def apply(self, z):
        return self.M @ z


def _whitened_operator(n, eta, seed):
    rng = np.random.default_rng(seed)
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = rng.uniform(1 / (1 + eta), 1 / (1 - eta), size=n)
    s[0], s[-1] = 1 / (1 + eta), 1 / (1 - eta)
    return (Q1 * s ** 2) @ Q1.T


@pytest.mark.parametrize("eta", [0.2887, 0.5])
def test_polyak_contraction_bound(eta):
    n = 40
    M = _whitened_operator(n, eta, 1)
    c = np.random.default_rng(2).standard_normal(n)
    exact = np.linalg.solve(M, c)
    beta = eta ** 2
    alpha = (1 - beta) ** 2
    for k in range(1, 40):
        dy, used = O._polyak(_Op(M), c, alpha, beta, k, None)
        assert used == k
        j = k + 1                       # dy_(j) after k updates (Alg. 5 indexing)
        bound = 4 * math.sqrt(2) * j * eta ** (j - 2) * np.linalg.norm(c)
        assert np.linalg.norm(dy - exact) <= bound + 1e-13 * np.linalg.norm(exact)


def test_polyak_identity_special_case():
    n = 10
    c = np.random.default_rng(3).standard_normal(n)
    dy, _ = O._polyak(_Op(np.eye(n)), c, 1.0, 0.0, 1, None)
    assert np.array_equal(dy, c)


def test_cg_finite_termination():
    n = 8
    M = _whitened_operator(n, 0.9, 4)
    c = np.random.default_rng(5).standard_normal(n)
    dy, _ = O._cg(_Op(M), c, n - 1, None)
    assert np.linalg.norm(M @ dy - c) >= 1e-6 * np.linalg.norm(c)   # not yet
    dy, _ = O._cg(_Op(M), c, n, None)
    # exact arithmetic gives zero after n steps; kappa(M) = 361 leaves ~1e-11
    assert np.linalg.norm(M @ dy - c) <= 1e-9 * np.linalg.norm(c)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("method", ["fossils", "spir"])
def test_solver_backward_stable_config1(method, seed):
    P = problem_svd(4000, 50, 1e12, 1e-6, seed=seed)
    A, b, xt = P["A"], P["b"], P["x_true"]
    x_qr, R_A = O.qr_solve(A, b, return_R=True)
    res = getattr(O, method)(A, b, seed=seed)
    be = O.kw_relative(A, b, res["x"], R_A=R_A)
    assert be <= 1e-13
    assert O.forward_error(res["x"], xt) <= 10 * O.forward_error(x_qr, xt)
    # one refinement step is forward but not backward stable on this
    # large-residual, ill-conditioned problem (Sec. 5.1)
    be1 = O.kw_relative(A, b, res["iterates"][1], R_A=R_A)
    assert be1 > 10 * be


def test_table2_norm_c():
    gold = json.load(open(os.path.join(GOLDEN, "table2_norm_c.json")))
    vals = {"zero_init": [], "sketch_and_solve_x0": [], "strongly_forward_stable_x1": []}
    for seed in range(5):
        P = problem_svd(gold["m"], gold["n"], gold["kappa"], gold["resid_norm"], seed=seed)
        pr = O._Problem(P["A"], P["b"], None, 8, seed, None, True)
        c0, _ = pr.rhs(np.zeros(gold["n"]))
        vals["zero_init"].append(np.linalg.norm(c0))
        res = O.fossils(P["A"], P["b"], seed=seed)
        vals["sketch_and_solve_x0"].append(res["cnorms"][0])
        vals["strongly_forward_stable_x1"].append(res["cnorms"][1])
    for k, paper in gold["norm_c"].items():
        med = float(np.median(vals[k]))
        assert paper / 10 <= med <= paper * 10, (k, med, paper)


def test_table1_residual_orthogonality():
    gold = json.load(open(os.path.join(GOLDEN, "table1_residual_orthogonality.json")))
    orth = {"fossils": [], "spir": []}
    for seed in range(9):
        P = problem_svd(gold["m"], gold["n"], gold["kappa"], gold["resid_norm"], seed=100 + seed)
        A, b = P["A"], P["b"]
        for k in orth:
            x = getattr(O, k)(A, b, seed=seed)["x"]
            _, _, g = O.residual_dot2(A, b, x)
            orth[k].append(np.linalg.norm(g))
    for k in orth:
        med = float(np.median(orth[k]))
        paper = gold["median_orthogonality"][k]
        assert paper / 10 <= med <= paper * 10, (k, med, paper)
        # and far below the strongly-forward-stable methods' level
        assert med < gold["median_orthogonality"]["iterative_sketching_momentum"] / 100


@pytest.mark.parametrize("theta", [None, 0.3])
def test_kw_closed_form(theta):
    P = problem_svd(3000, 20, 1e6, 1e-5, seed=6)
    A, b, U, s, V = P["A"], P["b"], P["U"], P["sigma"], P["V"]
    xhat = P["x_true"] + 1e-7 * np.random.default_rng(7).standard_normal(20)
    est = O.kw_estimate(A, b, xhat, theta=theta)
    th = np.linalg.norm(A) / np.linalg.norm(b) if theta is None else theta
    r_hi, r_lo, _ = O.residual_dot2(A, b, xhat)
    r = r_hi + r_lo
    nx = np.linalg.norm(xhat)
    lam = th ** 2 * np.linalg.norm(r) ** 2 / (1 + th ** 2 * nx ** 2)
    comp = s * (U.T @ r)                  # A^T r in the V basis
    closed = th / math.sqrt(1 + th ** 2 * nx ** 2) * math.sqrt(float(np.sum(comp ** 2 / (s ** 2 + lam))))
    assert abs(est - closed) <= 1e-6 * closed


def test_kw_below_perturbation():
    """BE-hat <= BE <= ||Delta A||_F when x solves the perturbed problem."""
    rng = np.random.default_rng(9)
    m, n = 500, 8
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    dA = 1e-9 * rng.standard_normal((m, n))
    x = np.linalg.lstsq(A + dA, b, rcond=None)[0]
    est = O.kw_estimate(A, b, x, theta=1e8)
    assert est <= 1.05 * np.linalg.norm(dA)
    assert est >= 1e-3 * np.linalg.norm(dA)


def _preconditioned_problem(kappa, resid, seed, m=3000, n=30):
    """The preconditioned operator B = A D^{-1} R^{-1} of a constructed
    problem and a generic right-hand side r (a refinement residual is nearly
    orthogonal to range(A), so B^T r cancels heavily and its rounding would
    swamp the comparison), with c = B^T r."""
    P = problem_svd(m, n, kappa, resid, seed=seed)
    prob = O._Problem(P["A"], P["b"], None, 8, seed, None, True)
    r = np.random.default_rng(seed + 100).standard_normal(m)
    c = O.backsub_t(prob.R, prob.As.T @ r)
    return prob, c, r


@pytest.mark.parametrize("steps", [1, 3, 6])
def test_lsqr_iterates_match_cg(steps):
    """LSQR on min ||r - B dy|| and CG on B^T B dy = B^T r (B = A R^{-1}) give
    the same iterates in exact arithmetic.  With kappa(A) = 10 the triangular
    solves with R are accurate to rounding (their forward error grows with
    kappa(R)), so the two oracle solvers must agree to rounding."""
    prob, c, r = _preconditioned_problem(10.0, 1e-4, 3)
    dy_l, k_l = O._lsqr(prob, r, steps, None)
    dy_c, k_c = O._cg(prob, c, steps, None)
    assert k_l == k_c == steps
    assert np.linalg.norm(dy_l - dy_c) <= 1e-11 * np.linalg.norm(dy_c)


def test_lsqr_converges_to_least_squares_solution():
    """After enough steps LSQR's dy solves min ||r - B dy|| (LAPACK lstsq on
    the explicitly formed B as the reference)."""
    prob, c, r = _preconditioned_problem(1e4, 1e-2, 5, m=2000, n=20)
    dy, _ = O._lsqr(prob, r, 60, None)
    B = prob.As @ np.linalg.inv(prob.R)
    ref = np.linalg.lstsq(B, r, rcond=None)[0]
    assert np.linalg.norm(dy - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_spir_lsqr_backward_stable_config1(seed):
    """LSQR-based SPIR on Fig. 1's construction: backward stable after two
    steps, forward error within 10x of Householder QR, one step not enough;
    and (Sec. "SPIR: Conjugate gradient or LSQR?") its backward error is at
    the CG-based SPIR's level.  (The forward errors here are of order one for
    every solver, QR included, kappa = 1e12, so they are compared with QR's,
    not with each other's.)"""
    P = problem_svd(4000, 50, 1e12, 1e-6, seed=seed)
    A, b, xt = P["A"], P["b"], P["x_true"]
    x_qr, R_A = O.qr_solve(A, b, return_R=True)
    res = O.spir_lsqr(A, b, seed=seed)
    be = O.kw_relative(A, b, res["x"], R_A=R_A)
    assert be <= 1e-13
    fe = O.forward_error(res["x"], xt)
    assert fe <= 10 * O.forward_error(x_qr, xt)
    assert O.kw_relative(A, b, res["iterates"][1], R_A=R_A) > 10 * be
    cg = O.spir(A, b, seed=seed)
    be_cg = O.kw_relative(A, b, cg["x"], R_A=R_A)
    assert be <= max(10 * be_cg, 1e-15) and be_cg <= max(10 * be, 1e-15)
    assert res["iters"] == cg["iters"]   # the same stopping decisions


def test_sketched_kw_without_sketch_is_kw():
    """With SA replaced by A itself (no sketch, distortion 0) the sketched
    estimate (eq. (sketched-kw), through the SVD) is the Karlson-Walden
    estimate (through a QR), so the two routes agree to rounding."""
    P = problem_svd(2000, 30, 1e6, 1e-3, seed=8)
    A, b = P["A"], P["b"]
    x = O.qr_solve(A, b) + 1e-9 * np.random.default_rng(1).standard_normal(30)
    kw = O.kw_estimate(A, b, x)
    sk = O.sketched_kw(A, A, b, x)
    assert abs(sk - kw) <= 1e-10 * kw


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sketched_kw_within_proposition_bounds(seed):
    """Proposition (sketched KW) with Fact (KW estimate): for an embedding of
    distortion eta, KW / (sqrt(2)(1 + eta)) <= BE_sk <= sqrt(2) KW / (1 - eta);
    checked with eta = 1/2 (d = 12n, zeta = 8 sparse sign) at perturbed
    solutions of several quality levels."""
    P = problem_svd(3000, 40, 1e8, 1e-4, seed=seed)
    A, b = P["A"], P["b"]
    SA, _ = O.sketch(A, b, 480, 8, seed)
    eta = 0.5
    x_qr = O.qr_solve(A, b)
    rng = np.random.default_rng(seed)
    for scale in (0.0, 1e-12, 1e-6):
        x = x_qr + scale * rng.standard_normal(40)
        kw = O.kw_estimate(A, b, x)
        sk = O.sketched_kw(SA, A, b, x)
        assert kw / (math.sqrt(2) * (1 + eta)) <= sk <= math.sqrt(2) * kw / (1 - eta)


@pytest.mark.parametrize("seed", [0, 1])
def test_fossils_sketched_kw_stop(seed):
    """Alg. 4's step-2 test: checks after updates 1, 6, 11, ...; where it
    stops, the estimate is below u ||A||_F (u = 2^-52) and the solution is
    backward stable.  It stops before Theorem 7.1's count on these
    problems."""
    P = problem_svd(4000, 50, 1e12, 1e-6, seed=seed)
    A, b = P["A"], P["b"]
    _, R_A = O.qr_solve(A, b, return_R=True)
    res = O.fossils(A, b, seed=seed, kw_stop=True)
    k2 = res["iters"][1]
    assert k2 < 100 and (k2 - 1) % 5 == 0
    assert O.kw_relative(A, b, res["x"], R_A=R_A) <= 1e-13
    As = A / O.column_norms(A)
    SA, _ = O.sketch(As, b, 600, 8, seed)
    xs = res["x"] * O.column_norms(A)   # (x / d) d: a rounding away from the x tested
    assert O.sketched_kw(SA, As, b, xs) < 1.1 * 2.0 ** -52 * np.linalg.norm(As)
    assert k2 <= res["q2"]
