"""GPU parity of each step of the hot path against the CPU oracle, through
the C ABI (paper_2406_03468_gb300 is a ctypes binding of liblsq.so).

Sizes span several CTAs and row blocks with ragged tails (m = 20011 rows,
n = 130 or 37 columns, lda > n).  Bars:
  * sketch pattern: bit-exact (index work);
  * fixed-point sketch sums (m n >= 2^24): bit-exact (integer work);
  * other sums (scatter sketch, passes): within the standard summation error bound
    gamma_k sum |terms| with k the number of terms, written per element;
  * QR / triangular solves: normwise backward-error level, kappa(R) u.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2406_03468_gb300 as lsq
from gpu_util import DEV, H, T, empty
from lsq_problems import problem_gaussian, problem_svd
from oracle.philox import sparse_sign_matrix, sparse_sign_pattern

pytestmark = pytest.mark.gpu
u = 2.0 ** -53


@pytest.mark.parametrize("m,n,d,zeta,seed", [
    (20011, 50, 600, 8, 3),        # the paper's d = 12n, zeta = 8
    (3000, 4, 10, 8, 5),           # heavy rejection sampling
    (1000, 4, 8, 8, 1),            # d = zeta: every row of S hit
    (5000, 4, 37, 3, 2 ** 63 + 5),
    (777, 2, 5, 1, 0),
])
def test_pattern_bit_exact(m, n, d, zeta, seed):
    plan = lsq.Plan(m, n, d=d, zeta=zeta, seed=seed)
    rows = empty(m * zeta, torch.int32)
    sb = empty(m, torch.int32)
    lsq.lsq_sketch_pattern(plan.handle, rows, sb)
    r_or, s_or = sparse_sign_pattern(m, d, zeta, seed)
    assert np.array_equal(H(rows).reshape(m, zeta), r_or)
    bits = H(sb).view(np.uint32).astype(np.uint64)
    neg = (bits[:, None] >> np.arange(zeta, dtype=np.uint64)[None, :]) & np.uint64(1)
    assert np.array_equal(np.where(neg == 1, -1.0, 1.0), s_or)


def _problem(m, n, kappa, seed, lda=None):
    P = problem_svd(m, n, kappa, 1e-4, seed=seed, keep_factors=False)
    A = P["A"]
    if lda is not None and lda > n:
        Af = np.zeros((m, lda))
        Af[:, :n] = A
        Af[:, n:] = np.nan          # padding must never be read
        return P, Af
    return P, A


@pytest.mark.parametrize("m,n,lda", [(20011, 130, None), (20011, 37, None), (9001, 64, 70)])
def test_sketch_and_column_norms(m, n, lda):
    P, Afull = _problem(m, n, 1e3, seed=1, lda=lda)
    A, b = P["A"], P["b"]
    plan = lsq.Plan(m, n, lda=(lda or 0), seed=11)
    lsq.lsq_sketch(plan.handle, T(Afull), T(b))
    d = 12 * n
    SAb = empty(d * (n + 1))
    cn = empty(n)
    lsq.lsq_get_sketch(plan.handle, SAb, cn)
    SAb = H(SAb).reshape(n + 1, d).T
    dcol = oracle.column_norms(A)
    assert np.allclose(H(cn), dcol, rtol=1e-13, atol=0)
    SA, Sb = oracle.sketch(A / dcol, b, d, 8, 11)
    S = abs(sparse_sign_matrix(m, d, 8, 11))
    k = int(S.sum(axis=1).max() * math.sqrt(8)) + 2       # terms per sketch entry
    bound_A = (S @ np.abs(A / dcol)) * (k * u) * 4 + 1e-300
    bound_b = (S @ np.abs(b)) * (k * u) * 4 + 1e-300
    assert (np.abs(SAb[:, :n] - SA) <= bound_A).all()
    assert (np.abs(SAb[:, n] - Sb) <= bound_b).all()


@pytest.mark.parametrize("m,n", [(20011, 130), (4000, 50), (3001, 7), (60000, 500), (13001, 1000),
                                 (13001, 1024)])
def test_qr_of_sketch(m, n):
    P, A = _problem(m, n, 1e3, seed=2)
    plan = lsq.Plan(m, n, seed=4)
    lsq.lsq_sketch(plan.handle, T(A), T(P["b"]))
    d = 12 * n
    SAb = empty(d * (n + 1))
    lsq.lsq_get_sketch(plan.handle, SAb, None)
    SAb = H(SAb).reshape(n + 1, d).T
    R = empty(n * n)
    t = empty(n)
    x0 = empty(n)
    ce, ne = lsq.lsq_get_R(plan.handle, R, t, x0)
    R = H(R).reshape(n, n)
    R_or, V = oracle.householder_qr(SAb[:, :n])
    t_or = oracle.apply_qt(V, SAb[:, n])[:n]
    nR = np.linalg.norm(R_or, 2)
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.linalg.norm(R - R_or, 2) <= 1e3 * n * u * nR
    assert np.linalg.norm(H(t) - t_or) <= 1e3 * n * u * np.linalg.norm(SAb[:, n])
    # sketch-and-solve x0 = R^{-1} t: both R and t agree to rounding, so x0
    # agrees to kappa(R) times that (10 kappa(R) n u)
    x0_or = oracle.backsub(R_or, t_or)
    kR = np.linalg.cond(R_or)
    assert np.linalg.norm(H(x0) - x0_or) <= 10 * kR * n * u * np.linalg.norm(x0_or)
    # condest / normest against the exact singular values of R
    smax, smin = oracle.sigma_extremes(R_or)
    assert 0.7 * smax <= ne <= 1.0001 * smax
    # power iteration approaches the extreme singular values from inside
    assert 0.8 * smax / smin <= ce <= 1.0001 * smax / smin


@pytest.mark.parametrize("n", [37, 96, 97, 130, 500, 1024])
def test_triangular_solves(n):
    """n <= 96: one CTA; n > 96: the 8-CTA cluster form (n = 97: a last
    block of one row; n = 1024: 32 blocks, the most the update CTAs hold)."""
    P, A = _problem(20011, n, 1e6, seed=3)
    plan = lsq.Plan(20011, n, seed=5)
    lsq.lsq_sketch(plan.handle, T(A), T(P["b"]))
    R = empty(n * n)
    lsq.lsq_get_R(plan.handle, R)
    R = H(R).reshape(n, n)
    y = np.random.default_rng(0).standard_normal(n)
    for trans in (0, 1):
        out = empty(n)
        lsq.lsq_trsv(plan.handle, trans, T(y), out)
        ref = oracle.backsub(R, y) if trans == 0 else oracle.backsub_t(R, y)
        # backward stable solve: residual at the level n u |R| |x|
        Rop = R if trans == 0 else R.T
        res = np.abs(Rop @ H(out) - y)
        assert (res <= 4 * n * u * (np.abs(Rop) @ np.abs(H(out))) + 1e-300).all()
        kap = np.linalg.cond(R)
        assert np.linalg.norm(H(out) - ref) <= 10 * n * kap * u * np.linalg.norm(ref)


@pytest.mark.parametrize("m,n,lda", [(20011, 130, None), (20011, 37, None), (9001, 64, 70),
                                     (4097, 1000, None), (333, 1, None)])
def test_fused_passes(m, n, lda):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    Afull = A
    if lda:
        Afull = np.full((m, lda), np.nan)
        Afull[:, :n] = A
    z = rng.standard_normal(n)
    b = rng.standard_normal(m)
    plan = lsq.Plan(m, n, lda=(lda or 0), seed=1)
    dA = T(Afull)
    h = empty(n)
    lsq.lsq_apply_normal(plan.handle, dA, T(z), h)
    t_ref = A @ z
    h_ref = A.T @ t_ref
    bound = 4 * (n + m) * u * (np.abs(A).T @ (np.abs(A) @ np.abs(z)))
    assert (np.abs(H(h) - h_ref) <= bound).all()
    # residual pass against the compensated oracle
    g = empty(n)
    r2 = lsq.lsq_residual(plan.handle, dA, T(b), T(z), g)
    r_hi, r_lo, g_ref = oracle.residual_dot2(A, b, z)
    bound = 4 * (n + m) * u * (np.abs(A).T @ (np.abs(b) + np.abs(A) @ np.abs(z)))
    assert (np.abs(H(g) - g_ref) <= bound).all()
    assert abs(r2 - float(r_hi @ r_hi)) <= 1e-12 * float(r_hi @ r_hi)


def test_invalid_inputs():
    m, n = 500, 10
    rng = np.random.default_rng(1)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    x = empty(n)
    plan = lsq.Plan(m, n)
    Abad = A.copy()
    Abad[7, 3] = np.nan
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_solve_fossils(plan.handle, T(Abad), T(b), x)
    assert e.value.status == -6
    bbad = b.copy()
    bbad[0] = np.inf
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_solve_spir(plan.handle, T(A), T(bbad), x)
    assert e.value.status == -6
    Az = A.copy()
    Az[:, 4] = 0.0
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_solve_fossils(plan.handle, T(Az), T(b), x)
    assert e.value.status == -1
    with pytest.raises(lsq.LsqError):
        lsq.lsq_solve_fossils(plan.handle, None, T(b), x)
    # the plan still works after the errors
    st, info = lsq.lsq_solve_fossils(plan.handle, T(A), T(b), x)
    assert st == 0
    assert np.allclose(H(x), np.linalg.lstsq(A, b, rcond=None)[0], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("m,n,scale", [(20011, 130, 1.0), (20011, 37, 1.0), (4097, 1000, 1.0),
                                       (60000, 500, 1.0), (20011, 130, 2.0 ** 50)])
def test_inner_pass_fp32_pipe(m, n, scale):
    """The FP32-pipe inner passes against a compensated-arithmetic reference,
    on a z with 16 decades of dynamic range (as z = R^{-1} dy has on
    ill-conditioned problems), with the same per-element bound as the FP64
    pass.  scale 1: the double-float pass on the hi / lo planes; scale 2^50
    (outside the planes' range): the pass that splits A on the fly."""
    rng = np.random.default_rng(m + 3 * n)
    A = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-2, 2, n) * scale
    b = rng.standard_normal(m)
    z = rng.standard_normal(n) * 10.0 ** rng.uniform(-8, 8, n)
    out = {}
    for flag in (0, 1):
        plan = lsq.Plan(m, n, seed=1, inner_fp64_fma=flag)
        dA = T(A)
        lsq.lsq_sketch(plan.handle, dA, T(b))
        h = empty(n)
        lsq.lsq_apply_normal(plan.handle, dA, T(z), h)
        out[flag] = H(h)
        plan.close()
    _, _, h_ref = oracle.residual_dot2(A, np.zeros(m), -z)    # A^T (A z), compensated
    scale = np.abs(A).T @ (np.abs(A) @ np.abs(z))
    bound = 4 * (n + m) * u * scale
    for flag in (0, 1):
        assert (np.abs(out[flag] - h_ref) <= bound).all(), flag
    err_eft = float(np.max(np.abs(out[0] - h_ref) / scale))
    err_f64 = float(np.max(np.abs(out[1] - h_ref) / scale))
    print("max relative error: fp32-pipe %.3g  fp64 %.3g  (u = %.3g)" % (err_eft, err_f64, u))


def test_inner_kernel_choice_badly_scaled_columns():
    """Which inner pass runs: the double-float pass on the planes (3) while
    every column norm is in [2^-40, 2^40] (columns 2^30 apart included); the
    on-the-fly split (1) for a uniform 2^50 scale; the FP64 pass (0) when
    column norms are 2^50 apart.  Every solve is backward stable."""
    P = problem_svd(20000, 40, 1e6, 1e-5, seed=4)
    b = P["b"]
    A30 = P["A"].copy()
    A30[:, :20] *= 2.0 ** 30
    A50 = P["A"].copy()
    A50[:, :20] *= 2.0 ** 50
    for Am, expect in ((P["A"], 3), (A30, 3), (P["A"] * 2.0 ** 50, 1), (A50, 0)):
        plan = lsq.Plan(20000, 40, seed=2)
        x = empty(40)
        st, info = plan.solve(T(Am), T(b), x, "fossils")
        assert info["inner_kernel"] == expect
        assert oracle.kw_relative(Am, b, H(x)) <= 1e-13
        plan.close()


@pytest.mark.parametrize("m,n", [(20011, 130), (4097, 1000)])
def test_residual_pass_after_sketch(m, n):
    """The residual pass after lsq_sketch (the state a solve runs it in), on
    columns of mixed scale: g within the FP64 componentwise bound of the
    compensated oracle, ||r||^2 to 1e-12 relative."""
    rng = np.random.default_rng(m * 3 + n)
    A = rng.standard_normal((m, n)) * np.exp2(rng.integers(-8, 8, size=n))
    b = rng.standard_normal(m)
    x = rng.standard_normal(n)
    plan = lsq.Plan(m, n, seed=2)
    dA, db = T(A), T(b)
    lsq.lsq_sketch(plan.handle, dA, db)
    g = empty(n)
    r2 = lsq.lsq_residual(plan.handle, dA, db, T(x), g)
    r_hi, r_lo, g_ref = oracle.residual_dot2(A, b, x)
    bound = 4 * (n + m) * u * (np.abs(A).T @ (np.abs(b) + np.abs(A) @ np.abs(x)))
    assert (np.abs(H(g) - g_ref) <= bound).all()
    assert abs(r2 - float(r_hi @ r_hi)) <= 1e-12 * float(r_hi @ r_hi)


@pytest.mark.parametrize("m,n,entry", [(200003, 100, "device"), (400003, 200, "host"),
                                        (20011, 1000, "device")])
def test_gather_sketch_fixed_point(m, n, entry):
    """The gather form of the sketch (m n >= 2^24).  Its raw sums are integer
    work and must equal oracle.fixed_point_sketch bit for bit.  Each list entry is
    truncated to a multiple of 2^F with F = (E - 1022) + L - 63 (E the
    largest biased exponent of the column in the rows summed, L = max(10,
    bits of the longest list)), so an entry of S A is off by less than
    cnt_h 2^(L-62) max|A_:j| plus FP64 roundings of the sums.  The host
    entry copies A in row chunks (640 MB here: 5 chunks of >= 128 MB) and
    sketches each as it lands, one fixed-point scale per chunk.  n = 1000
    takes the column-norm and exponent pass in two column halves."""
    P = problem_svd(m, n, 1e6, 1e-4, seed=13, keep_factors=False)
    A, b = P["A"], P["b"]
    zeta, d, seed = 8, 12 * n, 17
    plan = lsq.Plan(m, n, seed=seed)
    if entry == "device":
        lsq.lsq_sketch(plan.handle, T(A), T(b))
        nch = 1
    else:
        xh = np.empty(n)
        st, _ = lsq.lsq_solve_host(plan.handle, 0, A, b, xh)
        assert st == 0
        nch = min(16, int(8.0 * A.size // 128e6))
        assert nch == 5
    SAb = empty(d * (n + 1))
    cn = empty(n)
    lsq.lsq_get_sketch(plan.handle, SAb, cn)
    raw = empty(d * (n + 1))
    lsq.lsq_get_sketch_raw(plan.handle, raw)
    plan.close()
    # integer work: the fixed-point sums, rounded once to FP64 per row chunk,
    # equal the oracle's bit for bit
    bounds = [m * c // nch for c in range(nch + 1)]
    ref_raw = oracle.fixed_point_sketch(A, b, d, zeta, seed, row_chunks=bounds)
    got_raw = H(raw).reshape(d, n + 1)
    assert np.array_equal(got_raw.view(np.uint64), ref_raw.view(np.uint64)), \
        int((got_raw != ref_raw).sum())
    SAb = H(SAb).reshape(n + 1, d).T
    SAg = SAb[:, :n] * H(cn)            # undo the column scaling (3 roundings)
    SA, Sb = oracle.sketch(A, b, d, zeta, seed)
    S = abs(sparse_sign_matrix(m, d, zeta, seed)).sign()
    cnt = np.asarray(S.sum(axis=1)).ravel()
    L = max(10, int(cnt.max()).bit_length())
    c = 1.0 / math.sqrt(zeta)
    k = (nch + 8) + int(cnt.max())
    trunc_A = c * cnt[:, None] * 2.0 ** (L - 62) * np.abs(A).max(axis=0)[None, :]
    trunc_b = c * cnt * 2.0 ** (L - 62) * np.abs(b).max()
    bound_A = trunc_A + k * u * c * np.asarray(S @ np.abs(A)) + 1e-300
    bound_b = trunc_b + k * u * c * np.asarray(S @ np.abs(b)).ravel() + 1e-300
    assert (np.abs(SAg - SA) <= bound_A).all(), np.max(np.abs(SAg - SA) / bound_A)
    assert (np.abs(SAb[:, n] - Sb) <= bound_b).all()


@pytest.mark.parametrize("m,n,k", [(40000, 200, 64), (20011, 130, 16), (9001, 256, 64),
                                   (5003, 37, 8)])
def test_multi_rhs_inner_pass(m, n, k):
    """The many-right-hand-side inner pass (every row block of A applied to all
    k vectors in one read of the hi / lo planes) against the oracle's
    compensated A^T (A z_c), per element, with the FP64 per-element bound, on
    vectors spanning 16 decades and columns of A spanning 4; ragged row
    blocks (m not a multiple of the block) and widths n not a multiple of 4.
    Then the same with the DMMA pass (inner_fp64_fma = 1)."""
    rng = np.random.default_rng(m + 7 * n + k)
    A = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-2, 2, n)
    B = rng.standard_normal((m, k))
    Z = rng.standard_normal((k, n)) * 10.0 ** rng.uniform(-8, 8, (k, n))   # vector c = Z[c]
    for fp64 in (0, 1):
        plan = lsq.Plan(m, n, seed=3, nrhs=k, inner_fp64_fma=fp64)
        dA = T(A)
        X = torch.empty((n, k), dtype=torch.float64, device="cuda")
        st, info = lsq.lsq_solve_fossils_multi(plan.handle, dA, T(B), k, X)
        assert info.inner_kernel == (4 if fp64 else 5)
        Hd = empty(n * k)
        lsq.lsq_apply_normal_multi(plan.handle, dA, T(np.ascontiguousarray(Z)), Hd)
        Hh = H(Hd).reshape(k, n)
        plan.close()
        absA = np.abs(A)
        for c in range(k):
            _, _, h_ref = oracle.residual_dot2(A, np.zeros(m), -Z[c])
            bound = 4 * (n + m) * u * (absA.T @ (absA @ np.abs(Z[c])))
            assert (np.abs(Hh[c] - h_ref) <= bound).all(), (fp64, c)


@pytest.mark.parametrize("m,n,seed", [(4000, 50, 0), (20011, 130, 3)])
def test_sketched_kw_estimate(m, n, seed):
    """lsq_sketched_kw (eq. (sketched-kw), through the QR of [R; sqrt(lam) I])
    against oracle.sketched_kw (through the SVD of SA), on the column-scaled
    problem of the same sketch: at perturbed solutions the two agree to
    1e-4 relative (the estimate is well above the residual's rounding), and
    at the least-squares solution both sit at the u ||A D^-1||_F level."""
    P = problem_svd(m, n, 1e10, 1e-6, seed=seed, keep_factors=False)
    A, b = P["A"], P["b"]
    plan = lsq.Plan(m, n, seed=seed + 1)
    dA, db = T(A), T(b)
    lsq.lsq_sketch(plan.handle, dA, db)
    dcol = oracle.column_norms(A)
    As = A / dcol
    SA, _ = oracle.sketch(As, b, 12 * n, 8, seed + 1)
    x_qr = oracle.qr_solve(A, b)
    rng = np.random.default_rng(seed)
    fro = math.sqrt(n)
    for scale in (1e-6, 1e-10, 0.0):
        x = x_qr * (1.0 + scale * rng.standard_normal(n))
        est = lsq.lsq_sketched_kw(plan.handle, dA, db, T(x))
        ref = oracle.sketched_kw(SA, As, b, x * dcol)
        if scale > 0:
            assert abs(est - ref) <= 1e-4 * ref, (scale, est, ref)
        else:
            assert est <= 10 * u * fro and ref <= 10 * u * fro, (est, ref)
    plan.close()
