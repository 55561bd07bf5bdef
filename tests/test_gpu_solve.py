"""End-to-end GPU FOSSILS and SPIR against the CPU oracle (C ABI).

Acceptance, on every result: Karlson-Walden backward error (Sec. 4.1,
theta = ||A||_F / ||b||, relative to ||A||_F) <= 1e-13, and forward error
within 10x of the oracle's Householder QR solve (against the known x_true
of the constructed problems; for the Gaussian-factor problems, whose
reference is the oracle QR solution itself, within 10x of the spread
between the oracle's own SPIR and QR solutions or of the first-order Wedin
bound, whichever is larger).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2406_03468_gb300 as lsq
from gpu_util import H, T, empty
from lsq_problems import csr_to_dense, problem_gaussian, problem_prony, problem_sparse, problem_svd

pytestmark = pytest.mark.gpu


def _gpu_solve(method, A, b, **opts):
    m, n = A.shape
    plan = lsq.Plan(m, n, **opts)
    x = empty(n)
    st, info = plan.solve(T(A), T(b), x, method)
    out = H(x)
    plan.close()
    return st, info, out


@pytest.mark.parametrize("method", ["fossils", "spir"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_config1_fig1_problem(method, seed):
    """4000 x 50, kappa = 1e12, ||r|| = 1e-6, d = 12n, zeta = 8 (Fig. 1)."""
    P = problem_svd(4000, 50, 1e12, 1e-6, seed=seed)
    A, b, xt = P["A"], P["b"], P["x_true"]
    st, info, x = _gpu_solve(method, A, b, seed=seed)
    assert st == 0
    x_qr, R_A = oracle.qr_solve(A, b, return_R=True)
    be = oracle.kw_relative(A, b, x, R_A=R_A)
    assert be <= 1e-13, (be, info)
    assert oracle.forward_error(x, xt) <= 10 * oracle.forward_error(x_qr, xt)
    ref = getattr(oracle, method)(A, b, seed=seed)
    # Step 1 stops at the first update below Alg. 4's threshold; which update
    # crosses it first depends on rounding order by a step or two.  Step 2
    # runs q0 - 1 updates on both sides (condest is estimated on the GPU,
    # exact in the oracle).
    assert abs(info["iters"][0] - ref["iters"][0]) <= 2, (info["iters"], ref["iters"])
    assert abs(info["iters"][1] - ref["iters"][1]) <= 1
    # ||c|| at x0 (Table 2: 3.0e-7) and at x1 (Table 2: 1.9e-11; rounding noise)
    assert ref["cnorms"][0] / 5 <= info["cnorm"][0] <= ref["cnorms"][0] * 5
    assert ref["cnorms"][1] / 10 <= info["cnorm"][1] <= ref["cnorms"][1] * 10


@pytest.mark.parametrize("method", ["fossils", "spir"])
def test_two_steps_needed(method):
    """x1 is forward but not backward stable on this large-residual,
    ill-conditioned problem; x2 is backward stable (Sec. 5.1)."""
    P = problem_svd(4000, 50, 1e12, 1e-3, seed=7)
    A, b = P["A"], P["b"]
    st1, _, x1 = _gpu_solve(method, A, b, seed=3, max_refine=1)
    st2, _, x2 = _gpu_solve(method, A, b, seed=3, max_refine=2)
    _, R_A = oracle.qr_solve(A, b, return_R=True)
    be1 = oracle.kw_relative(A, b, x1, R_A=R_A)
    be2 = oracle.kw_relative(A, b, x2, R_A=R_A)
    assert be2 <= 1e-13 and be1 > 10 * be2


@pytest.mark.parametrize("method", ["fossils", "spir"])
@pytest.mark.parametrize("m,n,kappa", [(200003, 500, 1e10), (50021, 130, 1e6)])
def test_config2_shape_reduced_m(method, m, n, kappa):
    """Config-2 generator (A = G/sqrt(m) diag(sigma) V^T, b = A x + 1e-4 g)."""
    P = problem_gaussian(m, n, kappa, 1e-4, seed=5)
    A, b = P["A"], P["b"]
    st, info, x = _gpu_solve(method, A, b, seed=9)
    assert st == 0
    x_qr, R_A = oracle.qr_solve(A, b, return_R=True)
    be = oracle.kw_relative(A, b, x, R_A=R_A)
    assert be <= 1e-13, (be, info)
    x_sp = oracle.spir(A, b, seed=9)["x"]
    spread = oracle.forward_error(x_sp, x_qr)
    r = b - A @ x_qr
    wed = oracle.wedin_bound(info["condest"], 1.0, x_qr, float(np.linalg.norm(r)))
    assert oracle.forward_error(x, x_qr) <= 10 * max(spread, wed), (oracle.forward_error(x, x_qr), spread, wed)


def test_host_entry_point_matches_device():
    P = problem_svd(6000, 64, 1e4, 1e-5, seed=3)
    A, b = P["A"], P["b"]
    plan = lsq.Plan(6000, 64, seed=2)
    x = empty(64)
    plan.solve(T(A), T(b), x, "fossils")
    xd = H(x)
    xh = np.empty(64)
    st, info = lsq.lsq_solve_host(plan.handle, 0, A, b, xh)
    assert st == 0
    assert np.linalg.norm(xh - xd) <= 1e-11 * np.linalg.norm(xd)
    assert oracle.kw_relative(A, b, xh) <= 1e-13


@pytest.mark.parametrize("method", [0, 1])
def test_host_entry_point_chunked(method):
    """300007 x 256 (614 MB of A): the host entry copies A in 4 row chunks
    and sketches each as it lands; the answer is backward stable and within
    10x of the oracle QR's forward error, like the device entry's."""
    m, n = 300007, 256
    P = problem_svd(m, n, 1e10, 1e-4, seed=31)
    A, b, xt = P["A"], P["b"], P["x_true"]
    plan = lsq.Plan(m, n, seed=6)
    xh = np.empty(n)
    st, info = lsq.lsq_solve_host(plan.handle, method, A, b, xh)
    assert st == 0
    x = empty(n)
    plan.solve(T(A), T(b), x, ("fossils", "spir")[method])
    xd = H(x)
    plan.close()
    x_qr, R_A = oracle.qr_solve(A, b, return_R=True)
    for xs in (xh, xd):
        assert oracle.kw_relative(A, b, xs, R_A=R_A) <= 1e-13
        assert oracle.forward_error(xs, xt) <= 10 * oracle.forward_error(x_qr, xt)


@pytest.mark.parametrize("m,n", [(64, 64), (1000, 1), (513, 33)])
def test_edge_shapes(m, n):
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    for method in ("fossils", "spir"):
        st, info, x = _gpu_solve(method, A, b, seed=1)
        assert st == 0
        assert oracle.kw_relative(A, b, x) <= 1e-13, (method, x[:4], info)


@pytest.mark.parametrize("m,n", [(1000, 1), (4000, 50), (6000, 100)])
def test_zero_rhs(m, n):
    """b = 0: the sketch-and-solve start, every residual and every inner
    right-hand side are exactly 0, so each method returns x = 0 exactly (CG
    stops before its first update, whose step would be 0 / 0)."""
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    b = np.zeros(m)
    for method in ("fossils", "spir", "spir_lsqr"):
        st, info, x = _gpu_solve(method, A, b, seed=2)
        assert st == 0, (method, info)
        assert np.all(x == 0.0), (method, x[:4], info)


@pytest.mark.parametrize("method", ["fossils", "spir"])
@pytest.mark.parametrize("kappa,path", [(1e4, lsq.LSQ_PREC_FP32_INNER), (1e10, lsq.LSQ_PREC_FP64)])
def test_fp32_tier_gate(method, kappa, path):
    """Config-5 construction at reduced m: with precision AUTO, kappa = 1e4
    takes the FP32-inner tier and kappa = 1e10 the all-FP64 path; both give
    a backward-stable x within 10x of the oracle QR's forward error."""
    P = problem_svd(60000, 500, kappa, 1e-4, seed=21)
    A, b, xt = P["A"], P["b"], P["x_true"]
    st, info, x = _gpu_solve(method, A, b, seed=4, precision=lsq.LSQ_PREC_AUTO)
    assert info["path"] == path, info
    x_qr, R_A = oracle.qr_solve(A, b, return_R=True)
    be = oracle.kw_relative(A, b, x, R_A=R_A)
    assert be <= 1e-13, (be, info)
    assert oracle.forward_error(x, xt) <= 10 * oracle.forward_error(x_qr, xt)
    if path == lsq.LSQ_PREC_FP32_INNER:
        assert info["inner_kernel"] == 2 and 2 <= info["refine_steps"] <= 6


def test_fp32_tier_forced_and_bytes():
    """FP32_INNER forces the tier; its inner passes stream half the bytes of
    the FP64 ones (bytes_a accounting: the sketch pass reads A and writes its
    hi / lo FP32 planes, each residual pass reads A, each tier pass the hi
    plane)."""
    P = problem_svd(30000, 130, 1e3, 1e-5, seed=22)
    A, b = P["A"], P["b"]
    st, info, x = _gpu_solve("fossils", A, b, seed=1, precision=lsq.LSQ_PREC_FP32_INNER)
    assert info["path"] == lsq.LSQ_PREC_FP32_INNER
    assert oracle.kw_relative(A, b, x) <= 1e-13
    mn8 = 8.0 * 30000 * 130
    steps = info["refine_steps"]
    resid_passes = steps + (1 if steps < 6 else 0)
    expect = 2.0 * mn8 + mn8 * resid_passes + 0.5 * mn8 * sum(info["iters"])
    assert abs(info["bytes_a"] - expect) <= 1e-9 * expect, (info["bytes_a"], expect, info)


_C5 = {}


def _config5_width_problem(kappa):
    """The 150000 x 1000 problem at this kappa and the oracle's QR solve of
    it, built once per kappa for both methods."""
    if kappa not in _C5:
        _C5.clear()
        P = problem_svd(150000, 1000, kappa, 1e-4, seed=51, keep_factors=False)
        x_qr, R_A = oracle.qr_solve(P["A"], P["b"], return_R=True)
        _C5[kappa] = (P, x_qr, R_A)
    return _C5[kappa]


@pytest.mark.parametrize("m,n", [(1000, 1), (4000, 50), (6000, 100)])
def test_zero_rhs(m, n):
    """b = 0: the sketch-and-solve start, every residual and every inner
    right-hand side are exactly 0, so each method returns x = 0 exactly (CG
    stops before its first update, whose step would be 0 / 0)."""
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    b = np.zeros(m)
    for method in ("fossils", "spir", "spir_lsqr"):
        st, info, x = _gpu_solve(method, A, b, seed=2)
        assert st == 0, (method, info)
        assert np.all(x == 0.0), (method, x[:4], info)


@pytest.mark.parametrize("method", ["fossils", "spir"])
@pytest.mark.parametrize("kappa,path", [(1e4, lsq.LSQ_PREC_FP32_INNER), (1e10, lsq.LSQ_PREC_FP64)])
def test_fp32_tier_config5_width(method, kappa, path):
    """Config 5's width, n = 1000 (150000 x 1000, the widest pass and QR
    instantiations): AUTO takes the FP32 tier at kappa = 1e4 and the FP64
    path at kappa = 1e10; both results are backward stable and within 10x of
    the oracle QR's forward error."""
    P, x_qr, R_A = _config5_width_problem(kappa)
    A, b, xt = P["A"], P["b"], P["x_true"]
    st, info, x = _gpu_solve(method, A, b, seed=8, precision=lsq.LSQ_PREC_AUTO)
    assert st == 0
    assert info["path"] == path, info
    if path == lsq.LSQ_PREC_FP32_INNER:
        assert info["inner_kernel"] == 2 and 2 <= info["refine_steps"] <= 6
    be = oracle.kw_relative(A, b, x, R_A=R_A)
    assert be <= 1e-13, (be, info)
    assert oracle.forward_error(x, xt) <= 10 * oracle.forward_error(x_qr, xt)


@pytest.mark.parametrize("fp64", [0, 1])
@pytest.mark.parametrize("m,n,k,kappa", [(40000, 200, 16, 1e8), (30011, 100, 8, 1e6),
                                         (20000, 200, 64, 1e8)])
def test_multi_rhs_shared_sketch(m, n, k, kappa, fp64):
    """k right-hand sides on one A (config-4 construction at reduced m), with
    the k-tiled double-float inner pass (default) and the DMMA one
    (inner_fp64_fma = 1): every column of X is backward stable and within
    10x of the oracle QR solution's Wedin-bound yardstick; the same column
    solved alone on the single-RHS path agrees to that level."""
    from lsq_problems import problem_multi_rhs
    P = problem_multi_rhs(m, n, k, kappa, 1e-5, seed=41)
    A, B = P["A"], P["B"]
    plan = lsq.Plan(m, n, seed=6, nrhs=k, inner_fp64_fma=fp64)
    X = torch.empty((n, k), dtype=torch.float64, device="cuda")
    st, info = lsq.lsq_solve_fossils_multi(plan.handle, T(A), T(B), k, X)
    assert st == 0
    assert info.inner_kernel == (4 if fp64 else 5)
    Xh = H(X)
    R_A, V = oracle.householder_qr(A)
    for c in range(k):
        b = B[:, c]
        x_qr = oracle.backsub(R_A, oracle.apply_qt(V, b)[:n])
        be = oracle.kw_relative(A, b, Xh[:, c], R_A=R_A)
        assert be <= 1e-13, (c, be)
        r = b - A @ x_qr
        wed = oracle.wedin_bound(kappa, 1.0, x_qr, float(np.linalg.norm(r)))
        assert oracle.forward_error(Xh[:, c], x_qr) <= 10 * max(wed, 1e-15), c
    plan.close()
    # column 0 alone through the single-RHS FOSSILS path
    st, info1, x0 = _gpu_solve("fossils", A, B[:, 0].copy(), seed=6)
    assert np.linalg.norm(x0 - Xh[:, 0]) <= 10 * max(wed, 1e-15) * np.linalg.norm(x0)


def test_multi_rhs_rejects_unsupported():
    with pytest.raises(lsq.LsqError):
        lsq.Plan(1000, 300, nrhs=8)       # n > 256
    with pytest.raises(lsq.LsqError):
        lsq.Plan(1000, 100, nrhs=12)      # not a multiple of 8


def test_plan_configure_retargets_without_allocation():
    plan = lsq.Plan(30000, 128, seed=1)
    for (m, n) in ((30000, 128), (12000, 40), (20000, 128)):
        P = problem_svd(m, n, 1e6, 1e-6, seed=m + n)
        lsq.lsq_plan_configure(plan.handle, lsq.lsq_options_default(m=m, n=n, seed=2))
        x = empty(n)
        st, info = lsq.lsq_solve_fossils(plan.handle, T(P["A"]), T(P["b"]), x)
        assert st == 0 and oracle.kw_relative(P["A"], P["b"], H(x)) <= 1e-13
    with pytest.raises(lsq.LsqError):
        lsq.lsq_plan_configure(plan.handle, lsq.lsq_options_default(m=40000, n=128))
    plan.close()


@pytest.mark.parametrize("method", ["fossils", "spir"])
@pytest.mark.parametrize("kappa", [1e0, 1e4, 1e8, 1e12])
@pytest.mark.parametrize("resid", [1e-12, 1e-6, 1e-1])
def test_difficulty_grid(method, kappa, resid):
    """The (kappa, ||r||) grid of the paper's stability experiments (Sec. 5,
    Fig. 1's construction at 4000 x 50): backward error <= 1e-13 at every
    point, and the forward error within 10x of the larger of the oracle QR
    solve's and the first-order Wedin bound (Fact 2.4)."""
    P = problem_svd(4000, 50, kappa, resid, seed=41)
    A, b, xt = P["A"], P["b"], P["x_true"]
    st, info, x = _gpu_solve(method, A, b, seed=12)
    assert st in (0, lsq.LSQ_WARN_RANK_DEFICIENT)
    x_qr, R_A = oracle.qr_solve(A, b, return_R=True)
    assert oracle.kw_relative(A, b, x, R_A=R_A) <= 1e-13, info
    wed = oracle.wedin_bound(kappa, 1.0, xt, resid)
    assert oracle.forward_error(x, xt) <= 10 * max(oracle.forward_error(x_qr, xt), wed)


@pytest.mark.parametrize("method", ["fossils", "spir"])
@pytest.mark.parametrize("kappa,resid", [(1e13, 1e-6), (1e14, 1e-2), (1e15, 1e-6)])
@pytest.mark.parametrize("fp64", [0, 1])
def test_high_condition(method, kappa, resid, fp64):
    """Fig. 1's construction (20000 x 100) up to kappa = 1e15, with the
    default double-float inner pass and with the all-FP64 pass: the
    backward error stays <= 1e-13.  At kappa = 1e15 the library flags the
    problem as numerically rank deficient (status 2) and still returns the
    answer."""
    P = problem_svd(20000, 100, kappa, resid, seed=3)
    A, b = P["A"], P["b"]
    st, info, x = _gpu_solve(method, A, b, seed=9, inner_fp64_fma=fp64)
    assert st in (0, lsq.LSQ_WARN_RANK_DEFICIENT)
    assert info["inner_kernel"] == (0 if fp64 else 3)
    _, R_A = oracle.qr_solve(A, b, return_R=True)
    assert oracle.kw_relative(A, b, x, R_A=R_A) <= 1e-13, info


def test_qr_wait_runs_out_and_plan_recovers():
    """A bounded device wait that runs out.  With qr_wait_us = 1 every CTA of
    the QR but the owner of column 0 waits for reflector 0, which takes the
    owner several microseconds to build; the waits give up, the solve
    returns LSQ_ERR_TIMEOUT (no hang, no fault), and the same plan,
    re-targeted with the default limit, solves the problem backward stably."""
    m, n = 60000, 500
    P = problem_svd(m, n, 1e6, 1e-4, seed=2, keep_factors=False)
    A, b = T(P["A"]), T(P["b"])
    plan = lsq.Plan(m, n, seed=3, qr_wait_us=1)
    x = empty(n)
    with pytest.raises(lsq.LsqError) as e:
        plan.solve(A, b, x, "fossils")
    assert e.value.status == -5, str(e.value)
    lsq.lsq_plan_configure(plan.handle, lsq.lsq_options_default(m=m, n=n, seed=3))
    st, info = plan.solve(A, b, x, "fossils")
    assert st == 0
    assert oracle.kw_relative(P["A"], P["b"], H(x)) <= 1e-13
    plan.close()


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("fp64", [0, 1])
def test_spir_lsqr_config1(seed, fp64):
    """LSQR-based SPIR (Sec. 4.2, "SPIR: conjugate gradient or LSQR?") on the
    Fig. 1 problem (4000 x 50, kappa = 1e12, ||r|| = 1e-6) against
    oracle.spir_lsqr: backward error <= 1e-13, forward error within 10x of
    the oracle QR solve's, the step-1 count within 2 of the oracle's (the
    first update below the threshold depends on rounding order), the
    step-2 count equal to q0 - 1 within 1, and ||c_0||, ||c_1|| at the
    oracle's level.  fp64 = 1: the LSQR passes in FP64 on A."""
    P = problem_svd(4000, 50, 1e12, 1e-6, seed=seed)
    A, b, xt = P["A"], P["b"], P["x_true"]
    st, info, x = _gpu_solve("spir_lsqr", A, b, seed=seed, inner_fp64_fma=fp64)
    assert st == 0
    x_qr, R_A = oracle.qr_solve(A, b, return_R=True)
    be = oracle.kw_relative(A, b, x, R_A=R_A)
    assert be <= 1e-13, (be, info)
    assert oracle.forward_error(x, xt) <= 10 * oracle.forward_error(x_qr, xt)
    ref = oracle.spir_lsqr(A, b, seed=seed)
    assert abs(info["iters"][0] - ref["iters"][0]) <= 2, (info["iters"], ref["iters"])
    assert abs(info["iters"][1] - ref["iters"][1]) <= 1
    assert ref["cnorms"][0] / 5 <= info["cnorm"][0] <= ref["cnorms"][0] * 5
    assert ref["cnorms"][1] / 10 <= info["cnorm"][1] <= ref["cnorms"][1] * 10


@pytest.mark.parametrize("m,n,kappa", [(200003, 500, 1e10), (50021, 130, 1e6)])
def test_spir_lsqr_config2_shape(m, n, kappa):
    """LSQR-based SPIR on the config-2 generator at reduced m: backward
    stable, and within 10x of the larger of the oracle's own LSQR-SPIR /
    QR spread and the first-order Wedin bound of the oracle QR solution."""
    P = problem_gaussian(m, n, kappa, 1e-4, seed=5)
    A, b = P["A"], P["b"]
    st, info, x = _gpu_solve("spir_lsqr", A, b, seed=9)
    assert st == 0
    x_qr, R_A = oracle.qr_solve(A, b, return_R=True)
    be = oracle.kw_relative(A, b, x, R_A=R_A)
    assert be <= 1e-13, (be, info)
    x_sp = oracle.spir_lsqr(A, b, seed=9)["x"]
    spread = oracle.forward_error(x_sp, x_qr)
    r = b - A @ x_qr
    wed = oracle.wedin_bound(info["condest"], 1.0, x_qr, float(np.linalg.norm(r)))
    assert oracle.forward_error(x, x_qr) <= 10 * max(spread, wed)


def test_spir_lsqr_host_entry_and_edges():
    """method 2 through the host-buffer entry point, and the edge shapes
    (square, one column, ragged) on the device entry."""
    P = problem_svd(6000, 64, 1e6, 1e-5, seed=4)
    A, b = P["A"], P["b"]
    plan = lsq.Plan(6000, 64, seed=2)
    xh = np.empty(64)
    st, info = lsq.lsq_solve_host(plan.handle, 2, A, b, xh)
    assert st == 0
    assert oracle.kw_relative(A, b, xh) <= 1e-13
    plan.close()
    for (m, n) in ((64, 64), (1000, 1), (513, 33)):
        rng = np.random.default_rng(m * 7 + n)
        A = rng.standard_normal((m, n))
        b = rng.standard_normal(m)
        st, info, x = _gpu_solve("spir_lsqr", A, b, seed=1)
        assert st == 0
        assert oracle.kw_relative(A, b, x) <= 1e-13


@pytest.mark.parametrize("method", ["fossils", "spir"])
@pytest.mark.parametrize("seed", [0, 1])
def test_kw_stop_step2(method, seed):
    """Alg. 4's step-2 test on the GPU (kw_stop = 1): the estimate is checked
    after updates 1, 6, 11, ...; where the oracle's test stops early on these
    Fig. 1 problems the GPU stops at a check too, within one check of the
    oracle's, with the estimate below u ||A D^-1||_F (u = 2^-52) and a
    backward-stable answer (step 2's inner passes are FP64 under the test)."""
    P = problem_svd(4000, 50, 1e12, 1e-6, seed=seed)
    A, b, xt = P["A"], P["b"], P["x_true"]
    st, info, x = _gpu_solve(method, A, b, seed=seed, kw_stop=1)
    assert st == 0
    k2 = info["iters"][1]
    assert k2 < 100 and (k2 - 1) % 5 == 0, info["iters"]
    assert info["be_sketch_est"] < 2.0 ** -52 * math.sqrt(50)
    x_qr, R_A = oracle.qr_solve(A, b, return_R=True)
    assert oracle.kw_relative(A, b, x, R_A=R_A) <= 1e-13
    assert oracle.forward_error(x, xt) <= 10 * oracle.forward_error(x_qr, xt)
    if method == "fossils":
        ref = oracle.fossils(A, b, seed=seed, kw_stop=True)
        assert abs(k2 - ref["iters"][1]) <= 5, (k2, ref["iters"])


@pytest.mark.parametrize("method", ["fossils", "spir", "spir_lsqr"])
@pytest.mark.parametrize("m,n", [(20000, 40), (6001, 300)])
def test_complex_prony(method, m, n):
    """Complex least squares (the Prony experiment's first solve, synthetic:
    Toeplitz A from noisy unit-modulus exponentials, condition ~1e6) through
    the real embedding on the GPU: the complex Karlson-Walden backward error
    <= 1e-13, the answer within 10x of the level LAPACK's complex solver and
    the oracle (the same method on the same embedding and sketch seed) reach,
    and the step counts of the oracle's run."""
    P = problem_prony(m, n, seed=7)
    A, b = P["A"], P["b"]
    code = {"fossils": 0, "spir": 1, "spir_lsqr": 2}[method]
    plan = lsq.Plan(2 * m, 2 * n, seed=5)
    dA = torch.from_numpy(A).cuda()
    db = torch.from_numpy(b).cuda()
    dx = torch.empty(n, dtype=torch.complex128, device="cuda")
    work = torch.empty(4 * m * n, dtype=torch.float64, device="cuda")
    st, info = lsq.lsq_solve_complex(plan.handle, code, dA, db, dx, work)
    assert st == 0
    info = info.as_dict()
    plan.close()
    x = dx.cpu().numpy()
    assert np.all(np.isfinite(x))
    assert oracle.kw_relative_complex(A, b, x) <= 1e-13, info
    xl = np.linalg.lstsq(A, b, rcond=None)[0]
    xo, ref = oracle.solve_complex(method, A, b, seed=5)
    e_l = np.linalg.norm(xo - xl) / np.linalg.norm(xl)
    e_g = np.linalg.norm(x - xl) / np.linalg.norm(xl)
    assert e_g <= 10 * max(e_l, 1e-14), (e_g, e_l)
    assert abs(info["iters"][0] - ref["iters"][0]) <= 2, (info["iters"], ref["iters"])
    assert abs(info["iters"][1] - ref["iters"][1]) <= 1, (info["iters"], ref["iters"])


def test_complex_entry_errors():
    """Argument checks of the complex entry: odd plan sizes, lda < n and a
    misaligned A are refused before any launch; the plan then solves."""
    P = problem_prony(2000, 8, seed=1)
    A, b = P["A"], P["b"]
    dA, db = torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda()
    dx = torch.empty(8, dtype=torch.complex128, device="cuda")
    work = torch.empty(4 * 2000 * 8, dtype=torch.float64, device="cuda")
    odd = lsq.Plan(4000, 15, seed=1)
    with pytest.raises(lsq.LsqError):
        lsq.lsq_solve_complex(odd.handle, 0, dA, db, dx, work)
    odd.close()
    plan = lsq.Plan(4000, 16, seed=1)
    with pytest.raises(lsq.LsqError):
        lsq.lsq_solve_complex(plan.handle, 0, dA, db, dx, work, lda=4)
    with pytest.raises(lsq.LsqError):
        lsq.lsq_solve_complex(plan.handle, 0, dA.data_ptr() + 8, db, dx, work)
    st, _ = lsq.lsq_solve_complex(plan.handle, 0, dA, db, dx, work)
    assert st == 0
    assert oracle.kw_relative_complex(A, b, dx.cpu().numpy()) <= 1e-13
    plan.close()


def _csr_dev(P):
    return (torch.from_numpy(P["row_ptr"]).cuda(), torch.from_numpy(P["col"]).cuda(),
            torch.from_numpy(P["val"]).cuda(), torch.from_numpy(P["b"]).cuda())


@pytest.mark.parametrize("method", ["fossils", "spir", "spir_lsqr"])
@pytest.mark.parametrize("m,n,k,delta,d3", [(20011, 130, 8, None, False), (6001, 300, 20, 1e-8, False),
                                            (6001, 300, 20, 1e-8, True)])
def test_sparse_csr(method, m, n, k, delta, d3):
    """Sparse A (CSR; synthetic stand-in for the SuiteSparse runs, with SPIR's
    d = 3n in one case) on the GPU against the oracle on the same matrix
    densified: backward error <= 1e-13, forward error within 10x of the
    oracle QR solve's against x_true, and the oracle's step counts (same
    seed, so the same sketch pattern).  FOSSILS at d = 3n (eta = 0.58; the
    paper pairs d = 3n with SPIR) does not meet the step-1 threshold within
    100 updates at condition 3e8, in the oracle as on the GPU: there the GPU
    must match the oracle's counts and backward error (within 2x)."""
    P = problem_sparse(m, n, k, seed=3, delta=delta)
    A = csr_to_dense(P, m, n)
    b = P["b"]
    d = 3 * n if d3 else 0
    code = {"fossils": 0, "spir": 1, "spir_lsqr": 2}[method]
    plan = lsq.Plan(m, n, seed=5, sparse=1, d=d)
    rp, col, val, db = _csr_dev(P)
    dx = empty(n)
    st, info = lsq.lsq_solve_csr(plan.handle, code, rp, col, val, db, dx)
    info = info.as_dict()
    plan.close()
    assert st == 0
    x = H(dx)
    x_qr, R_A = oracle.qr_solve(A, b, return_R=True)
    ref = getattr(oracle, method)(A, b, seed=5, d=d or None)
    be = oracle.kw_relative(A, b, x, R_A=R_A)
    if method == "fossils" and d3:
        be_ref = oracle.kw_relative(A, b, ref["x"], R_A=R_A)
        assert ref["iters"][0] == 100 and be <= 2 * be_ref, (be, be_ref, info)
    else:
        assert be <= 1e-13, info
        xt = P["x_true"]
        assert oracle.forward_error(x, xt) <= 10 * max(oracle.forward_error(x_qr, xt), 1e-15)
    assert abs(info["iters"][0] - ref["iters"][0]) <= 2, (info["iters"], ref["iters"])
    assert abs(info["iters"][1] - ref["iters"][1]) <= 1, (info["iters"], ref["iters"])
    assert info["inner_kernel"] == 0


def test_sparse_csr_checks():
    """The CSR entry refuses a structure that is not CSR of m x n with nnz
    entries (a column index out of range, row_ptr[m] != nnz, a decreasing
    row_ptr) and NaN values before any pass reads them; a dense plan refuses
    CSR input and a sparse plan dense input; the plan then solves."""
    m, n, k = 3001, 40, 6
    P = problem_sparse(m, n, k, seed=9)
    rp, col, val, db = _csr_dev(P)
    dx = empty(n)
    plan = lsq.Plan(m, n, seed=1, sparse=1)
    bad = col.clone()
    bad[17] = n
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_solve_csr(plan.handle, 0, rp, bad, val, db, dx)
    assert e.value.status == -1
    badp = rp.clone()
    badp[m] -= 1
    with pytest.raises(lsq.LsqError):
        lsq.lsq_solve_csr(plan.handle, 0, badp, col, val, db, dx)
    badp = rp.clone()
    badp[5] = badp[7]
    with pytest.raises(lsq.LsqError):
        lsq.lsq_solve_csr(plan.handle, 0, badp, col, val, db, dx)
    nanv = val.clone()
    nanv[3] = float("nan")
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_solve_csr(plan.handle, 0, rp, col, nanv, db, dx)
    assert e.value.status == -6
    with pytest.raises(lsq.LsqError):
        lsq.lsq_solve_fossils(plan.handle, T(csr_to_dense(P, m, n)), db, dx)
    st, _ = lsq.lsq_solve_csr(plan.handle, 1, rp, col, val, db, dx)
    assert st == 0
    A = csr_to_dense(P, m, n)
    assert oracle.kw_relative(A, P["b"], H(dx)) <= 1e-13
    plan.close()
    dense = lsq.Plan(m, n, seed=1)
    with pytest.raises(lsq.LsqError):
        lsq.lsq_solve_csr(dense.handle, 0, rp, col, val, db, dx)
    dense.close()
