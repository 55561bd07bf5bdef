"""Served stream (continuous batching) through the C ABI: lsq_server_create /
lsq_submit / lsq_poll.

Problems shaped like the served configuration (uneven m, n in {32, 64, 128,
256}, kappa log-uniform in [1e2, 1e12], A = U diag(sigma) V^T,
b = A x + 1e-6 g) are solved alone (one plan each) and as a mix through a
server whose arena holds only part of them at once, so requests queue and
are admitted as slots and memory free up.  Each mixed result must be
backward stable (Karlson-Walden, <= 1e-13) and equal to its alone result
within 10x the first-order Wedin bound of the problem.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2406_03468_gb300 as lsq
from gpu_util import H, T, empty
from lsq_problems import problem_svd_torch

pytestmark = pytest.mark.gpu


def _stream(count, seed, m_lo=20000, m_hi=60000):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi))))
        n = int(rng.choice([32, 64, 128, 256]))
        kappa = 10.0 ** rng.uniform(2, 12)
        P = problem_svd_torch(m, n, kappa, 1e-6, seed=1000 + i)
        out.append({"m": m, "n": n, "kappa": kappa, "A": P["A"], "b": P["b"], "seed": 77 + i})
    return out


def test_alone_equals_mix():
    probs = _stream(16, seed=5)
    # alone
    for p in probs:
        plan = lsq.Plan(p["m"], p["n"], seed=p["seed"])
        x = empty(p["n"])
        st, info = plan.solve(p["A"], p["b"], x, "fossils")
        assert st in (0, 2)
        p["x_alone"] = H(x)
        plan.close()
    # mix: arena for about half of the total footprint
    foot = [8 * (p["m"] * p["n"] + p["m"] + p["n"]) + 3 * 256 for p in probs]
    arena = max(max(foot), sum(foot) // 2)
    srv = lsq.lsq_server_create(arena, 6, 60000, 256)
    tickets = []
    for p in probs:
        o = lsq.lsq_options_default(m=p["m"], n=p["n"], seed=p["seed"])
        tickets.append(lsq.lsq_submit(srv, o, 0, p["A"], p["b"], 1))
    pending = dict(zip(tickets, probs))
    while pending:
        for t in list(pending):
            p = pending[t]
            x = np.empty(p["n"])
            st, info, lat = lsq.lsq_poll(srv, t, x)
            if st == lsq.LSQ_PENDING:
                continue
            assert st in (0, 2)
            assert lat > 0
            p["x_mix"] = x
            del pending[t]
    stats = lsq.lsq_server_stats(srv)
    lsq.lsq_server_destroy(srv)
    assert stats["completed"] == len(probs) and stats["queued"] == 0
    assert stats["arena_peak"] <= arena < sum(foot)
    for p in probs:
        A = H(p["A"])
        b = H(p["b"])
        x_qr, R_A = oracle.qr_solve(A, b, return_R=True)
        assert oracle.kw_relative(A, b, p["x_mix"], R_A=R_A) <= 1e-13
        r = b - A @ x_qr
        wed = oracle.wedin_bound(p["kappa"], 1.0, x_qr, float(np.linalg.norm(r)))
        diff = np.linalg.norm(p["x_mix"] - p["x_alone"]) / np.linalg.norm(p["x_alone"])
        assert diff <= 10 * max(wed, 1e-15), (p["m"], p["n"], p["kappa"], diff, wed)


def test_admission_refusals():
    srv = lsq.lsq_server_create(1 << 20, 2, 10000, 64)     # 1 MiB arena
    A = torch.zeros((5000, 64), dtype=torch.float64, device="cuda")
    b = torch.zeros(5000, dtype=torch.float64, device="cuda")
    o = lsq.lsq_options_default(m=5000, n=64)                # 2.6 MB footprint > arena
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_submit(srv, o, 0, A, b, 1)
    assert e.value.status == -2
    o = lsq.lsq_options_default(m=20000, n=64)               # m > m_max
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_submit(srv, o, 0, A, b, 1)
    assert e.value.status == -1
    with pytest.raises(lsq.LsqError):
        lsq.lsq_poll(srv, 12345)
    lsq.lsq_server_destroy(srv)


def test_server_spir_and_host_buffers():
    P = problem_svd_torch(30000, 64, 1e8, 1e-6, seed=9)
    Ah, bh = H(P["A"]), H(P["b"])
    srv = lsq.lsq_server_create(64 << 20, 2, 40000, 128)
    o = lsq.lsq_options_default(m=30000, n=64, seed=3)
    t = lsq.lsq_submit(srv, o, 1, Ah, bh, 0)
    x = np.empty(64)
    while True:
        st, info, lat = lsq.lsq_poll(srv, t, x)
        if st != lsq.LSQ_PENDING:
            break
    lsq.lsq_server_destroy(srv)
    assert st == 0
    assert oracle.kw_relative(Ah, bh, x) <= 1e-13
