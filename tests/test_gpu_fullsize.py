"""Parity at the benchmark's full size and launch configuration: FOSSILS and
SPIR on the 1,000,000 x 500 FP64 problem A = (G/sqrt(m)) diag(sigma) V^T,
sigma log-spaced 1..1e-10, b = A x + 1e-4 g, d = 12n, zeta = 8 (the problem
bench.py times, same seeds, same plan options).

The oracle cannot run the whole method at this size in a test's time, so
the checks are the properties that hold at any size, computed by the oracle
on the GPU's answer:
  * Karlson-Walden backward error (Sec. 4.1) <= 1e-13, with the oracle's
    Householder R of A (O(m n^2) plain C, multi-threaded) and compensated
    residuals;
  * forward error against the oracle's Householder QR solution within 10x
    the first-order Wedin bound (Fact 2.4) with the GPU's condest;
  * residual orthogonality ||A^T (b - A x)|| no worse than 10x the oracle QR
    solution's (Sec. 1.1, Table 1's measure);
  * the step-2 count equals q0 - 1 of Theorem 7.1 at the GPU's condest.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2406_03468_gb300 as lsq
from lsq_problems import problem_gaussian

pytestmark = pytest.mark.gpu

M, N, KAPPA, NOISE, SEED, SKETCH_SEED = 1_000_000, 500, 1e10, 1e-4, 5, 9


@pytest.fixture(scope="module")
def full_problem():
    P = problem_gaussian(M, N, KAPPA, NOISE, seed=SEED)
    x_qr, R_A = oracle.qr_solve(P["A"], P["b"], return_R=True)
    _, _, g_qr = oracle.residual_dot2(P["A"], P["b"], x_qr)
    return P, x_qr, R_A, float(np.linalg.norm(g_qr))


@pytest.mark.parametrize("method", ["fossils", "spir"])
def test_full_size(full_problem, method):
    P, x_qr, R_A, orth_qr = full_problem
    A, b = P["A"], P["b"]
    plan = lsq.Plan(M, N, seed=SKETCH_SEED, timing=1)
    dA = torch.from_numpy(A).cuda()
    db = torch.from_numpy(b).cuda()
    x = torch.empty(N, dtype=torch.float64, device="cuda")
    st, info = plan.solve(dA, db, x, method)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    plan.close()
    assert st == 0
    be = oracle.kw_relative(A, b, xh, R_A=R_A)
    assert be <= 1e-13, (be, info)
    r = b - A @ x_qr
    wed = oracle.wedin_bound(info["condest"], 1.0, x_qr, float(np.linalg.norm(r)))
    assert oracle.forward_error(xh, x_qr) <= 10 * wed
    _, _, g = oracle.residual_dot2(A, b, xh)
    assert np.linalg.norm(g) <= 10 * orth_qr
    eta = math.sqrt(N / (12 * N))
    assert abs(info["iters"][1] - oracle.step2_updates(info["condest"], eta)) <= 0
