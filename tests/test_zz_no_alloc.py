"""The allocation-free fused pass (lsq_apply_normal_noalloc) against the
plan-based lsq_apply_normal, both through the C ABI, and against the
oracle's compensated A^T (A z).

Callers that cannot allocate device memory (a framework that owns all GPU
memory through its own pool, a latency-critical loop that cannot afford
cudaMalloc's synchronisation) use the no-allocation entry point; it must
give the same h = A^T (A z) as the plan-based pass, call after call, even
though every call reuses the same library-owned scratch array.  This file
is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2406_03468_gb300 as lsq

pytestmark = pytest.mark.gpu
u = 2.0 ** -53


@pytest.mark.parametrize("m,n,lda", [(20011, 130, 130), (9001, 64, 70), (4097, 1000, 1000)])
def test_noalloc_matches_plan_pass_twice(m, n, lda):
    rng = np.random.default_rng(m + n)
    A = np.full((m, lda), np.nan)
    A[:, :n] = rng.standard_normal((m, n))
    dA = torch.from_numpy(A).cuda()
    plan = lsq.Plan(m, n, lda=lda, seed=1)
    An = A[:, :n]
    for call in range(2):
        z = rng.standard_normal(n)
        dz = torch.from_numpy(z).cuda()
        h_plan = torch.empty(n, dtype=torch.float64, device="cuda")
        h_free = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        lsq.lsq_apply_normal(plan.handle, dA, dz, h_plan)
        lsq.lsq_apply_normal_noalloc(dA, m, n, lda, dz, h_free)
        torch.cuda.synchronize()
        hp = h_plan.cpu().numpy()
        hf = h_free.cpu().numpy()
        # the same per-element bound the pass tests use, against the plan
        # pass and against the oracle's compensated A^T (A z)
        bound = 4 * (n + m) * u * (np.abs(An).T @ (np.abs(An) @ np.abs(z)))
        _, _, h_ref = oracle.residual_dot2(An, np.zeros(m), -z)
        assert np.isfinite(hf).all(), call
        assert (np.abs(hf - hp) <= bound).all(), call
        assert (np.abs(hf - h_ref) <= bound).all(), call
    plan.close()


def test_noalloc_rejects_too_wide():
    A = torch.zeros((4, 2048), dtype=torch.float64, device="cuda")
    z = torch.zeros(2048, dtype=torch.float64, device="cuda")
    h = torch.zeros(2048, dtype=torch.float64, device="cuda")
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_apply_normal_noalloc(A, 4, 2048, 2048, z, h)
    assert e.value.status == -1
    assert "LSQ_MAX_N" in str(e.value)
