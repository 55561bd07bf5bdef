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


def test_batched_server_alone_equals_mix():
    """The batched server (lsq_server_create_batched): a stream of uneven
    requests, submitted together so that they share lockstep batches, gives
    each request the answer it gets alone in a batch of one, within the
    forward-error level; every answer is backward stable."""
    from lsq_problems import problem_svd
    shapes = [(20011, 32, 1e3), (41000, 64, 1e8), (15000, 128, 1e5), (60000, 256, 1e10),
              (33000, 100, 1e12), (24000, 48, 1e2)]
    Ps = [problem_svd(m, n, k, 1e-6, seed=900 + i, keep_factors=False)
          for i, (m, n, k) in enumerate(shapes)]
    dev = [(T(P["A"]), T(P["b"])) for P in Ps]
    srv = lsq.lsq_server_create_batched(2 << 30, 2, 8, 80000, 256)
    tickets = []
    for i, (A, b) in enumerate(dev):
        o = lsq.lsq_options_default(m=A.shape[0], n=A.shape[1], seed=5 + i)
        tickets.append(lsq.lsq_submit(srv, o, i % 2, A, b, 1))
    xs = {}
    for i, t in enumerate(tickets):
        x = np.empty(shapes[i][1])
        while True:
            st, info, lat = lsq.lsq_poll(srv, t, x)
            if st != lsq.LSQ_PENDING:
                break
        assert st >= 0
        xs[i] = x
    # each alone
    for i, (A, b) in enumerate(dev):
        o = lsq.lsq_options_default(m=A.shape[0], n=A.shape[1], seed=5 + i)
        t = lsq.lsq_submit(srv, o, i % 2, A, b, 1)
        x = np.empty(shapes[i][1])
        while True:
            st, info, lat = lsq.lsq_poll(srv, t, x)
            if st != lsq.LSQ_PENDING:
                break
        assert st >= 0
        P = Ps[i]
        wed = oracle.wedin_bound(shapes[i][2], 1.0, P["x_true"], 1e-6)
        assert np.linalg.norm(x - xs[i]) <= 10 * max(wed, 1e-15) * np.linalg.norm(x), i
        assert oracle.kw_relative(P["A"], P["b"], xs[i]) <= 1e-13, i
    lsq.lsq_server_destroy(srv)
