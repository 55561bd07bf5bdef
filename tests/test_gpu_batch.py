"""Batched solves (lsq_batch_solve): many problems in lockstep, each phase
one launch over all of them, against the CPU oracle and against the
single-problem path (C ABI).

Every item must meet the acceptance bars of the single-problem path:
Karlson-Walden backward error (Sec. 4.1, relative to ||A||_F) <= 1e-13 and
forward error within 10x of the oracle Householder QR solve's (the items are
Fig. 1 constructions with known x); the step-2 count is q0 - 1 of Theorem 7.1
at the item's condest; and an item solved in a batch agrees with the same
problem solved alone on the plan path to the forward-error level.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2406_03468_gb300 as lsq
from gpu_util import H, T, empty
from lsq_problems import problem_svd

pytestmark = pytest.mark.gpu

SHAPES = [(20011, 32, 1e2), (45000, 64, 1e6), (30000, 100, 1e10), (80021, 128, 1e4),
          (12000, 200, 1e12), (60000, 256, 1e8), (25000, 37, 1e11), (150000, 130, 1e3)]


def _problems(shapes, seed0=100):
    return [problem_svd(m, n, k, 1e-6, seed=seed0 + i, keep_factors=False)
            for i, (m, n, k) in enumerate(shapes)]


@pytest.fixture(scope="module")
def batch():
    h = lsq.lsq_batch_create(16, 256, 2_000_000 * 64)
    yield h
    lsq.lsq_batch_destroy(h)


@pytest.mark.parametrize("methods", [(0,) * 8, (1,) * 8, (0, 1, 1, 0, 1, 0, 0, 1)])
def test_batch_against_oracle(batch, methods):
    Ps = _problems(SHAPES)
    dev = [(T(P["A"]), T(P["b"]), empty(P["A"].shape[1])) for P in Ps]
    seeds = [7 + i for i in range(len(Ps))]
    st, stats, infos = lsq.lsq_batch_solve(batch, dev, seeds=seeds, methods=methods)
    assert st >= 0 and all(s >= 0 for s in stats), (st, stats)
    for i, P in enumerate(Ps):
        A, b, xt = P["A"], P["b"], P["x_true"]
        x = H(dev[i][2])
        x_qr, R_A = oracle.qr_solve_lapack(A, b, return_R=True)
        be = oracle.kw_relative(A, b, x, R_A=R_A)
        assert be <= 1e-13, (i, be, infos[i].as_dict())
        assert oracle.forward_error(x, xt) <= 10 * oracle.forward_error(x_qr, xt), i
        inf = infos[i]
        n = A.shape[1]
        eta = np.sqrt(n / (12.0 * n))
        assert inf.iters[1] == oracle.step2_updates(inf.condest, eta), (i, inf.iters[1])
        assert 1 <= inf.iters[0] < 100


def test_batch_matches_single_path(batch):
    """Each item against the same problem solved alone on the plan path
    (same sketch seed): the two differ only in summation order, so they agree
    to the forward-error level of the problem."""
    shapes = SHAPES[:5]
    Ps = _problems(shapes, seed0=300)
    dev = [(T(P["A"]), T(P["b"]), empty(P["A"].shape[1])) for P in Ps]
    seeds = [11 * (i + 1) for i in range(len(Ps))]
    st, stats, infos = lsq.lsq_batch_solve(batch, dev, seeds=seeds)
    assert st >= 0
    for i, P in enumerate(Ps):
        m, n = P["A"].shape
        plan = lsq.Plan(m, n, seed=seeds[i])
        xa = empty(n)
        plan.solve(dev[i][0], dev[i][1], xa, "fossils")
        plan.close()
        xb, xs = H(dev[i][2]), H(xa)
        kappa = shapes[i][2]
        wed = oracle.wedin_bound(kappa, 1.0, P["x_true"], 1e-6)
        assert np.linalg.norm(xb - xs) <= 10 * max(wed, 1e-15) * np.linalg.norm(xs), i


def test_batch_item_failure_is_isolated(batch):
    """A non-finite item reports LSQ_ERR_NONFINITE; the others still solve."""
    Ps = _problems(SHAPES[:3], seed0=500)
    Abad = Ps[1]["A"].copy()
    Abad[17, 3] = np.nan
    dev = [(T(Ps[0]["A"]), T(Ps[0]["b"]), empty(32)), (T(Abad), T(Ps[1]["b"]), empty(64)),
           (T(Ps[2]["A"]), T(Ps[2]["b"]), empty(100))]
    st, stats, infos = lsq.lsq_batch_solve(batch, dev, seeds=[1, 2, 3])
    assert stats[1] == -6 and st == -6
    for i in (0, 2):
        assert stats[i] >= 0
        assert oracle.kw_relative(Ps[i]["A"], Ps[i]["b"], H(dev[i][2])) <= 1e-13


def test_batch_rejects_bad_arguments(batch):
    A = torch.zeros((10, 300), dtype=torch.float64, device="cuda")
    b = torch.zeros(10, dtype=torch.float64, device="cuda")
    x = torch.zeros(300, dtype=torch.float64, device="cuda")
    with pytest.raises(lsq.LsqError):
        lsq.lsq_batch_solve(batch, [(A, b, x)])          # n > n_max, m < n


def test_batch_repeated_calls_and_sizes(batch):
    """The captured phases are reused across calls of the same shape class
    and re-captured for others; every call stays correct."""
    for rep, shapes in enumerate((SHAPES[:4], SHAPES[:4], SHAPES[2:7], SHAPES[:1])):
        Ps = _problems(shapes, seed0=700 + 10 * rep)
        dev = [(T(P["A"]), T(P["b"]), empty(P["A"].shape[1])) for P in Ps]
        st, stats, infos = lsq.lsq_batch_solve(batch, dev, seeds=list(range(len(Ps))))
        assert st >= 0
        for i, P in enumerate(Ps):
            assert oracle.kw_relative(P["A"], P["b"], H(dev[i][2])) <= 1e-13, (rep, i)
