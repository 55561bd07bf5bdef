"""Oracle: plain, slow, CPU FP64 reference for FOSSILS and SPIR.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg may import this module.  It shares no code with
the CUDA library and never calls it.

Every function names the passage of Epperly, Meier, Nakatsukasa,
"Fast randomized least-squares solvers can be just as accurate and stable as
classical direct solvers" (arXiv 2406.03468) that it follows.  Heavy loops
(Householder QR, triangular solves, compensated residuals) are plain C in
oracle/liboracle.c; matrix-vector products with A use numpy (a library
matvec serving as a step); sums are never blocked, fused or reordered beyond
what the definition states.

Readings of the paper that this oracle takes (the CUDA path takes the same ones):
  * u = 2^-53 (unit roundoff of IEEE double, the standard model of Sec. 1.4).
  * alpha, beta from eta = sqrt(n/d) (Sec. 4.2), i.e. beta = eta^2,
    alpha = (1 - beta)^2 (Sec. 2.3, optimal coefficients); Alg. 4's "beta <- d/n" is read as n/d.
  * normest = sigma_max(R), condest = sigma_max(R)/sigma_min(R): with a QR
    preconditioner the singular values of R equal those of SA, which Alg. 4
    reads off the SVD.
  * Step-1 stop (Sec. 4.2, "Adaptive stopping", item 1): stop after the first
    update Delta with ||Delta|| <= u (gamma normest ||x_0|| +
    rho condest ||b - A x_0||), at most 100 updates.  The text quotes
    gamma = 1, rho = 0.04; Alg. 4 uses 10 and 0.4.  The default is Alg. 4's:
    with the text's constants the threshold sits at the rounding-noise floor
    of ||Delta|| on ill-conditioned problems, where the update that first
    crosses it is a matter of rounding order (or never comes).
  * Step-2 count: q0 of Theorem 7.1 (Sec. 7) with kappa replaced by condest and the
    distortion 1.01 eta; Alg. 5 returns the iterate dy_(q) after q - 1 updates,
    so step 2 runs ceil(q0) - 1 updates (capped at 100).
  * SPIR's CG starts from dy = 0 and uses the same two stopping rules, with
    Delta = gamma_k p_k the CG update of dy.
  * Alg. 4's step-2 test reads "Mod(i, 5)" with i the refinement index, which
    is 1 throughout step 2; it is read as the inner index j: the sketched
    KW estimate is checked after updates 1, 6, 11, ... of the second solve.
  * The step-2 test's bound u ||A||_F takes u at the value Sec. 1.4 states
    for double precision, about 2e-16, i.e. 2^-52 (KW_STOP_U): at 2^-53 the
    bound sits at the estimate of the correctly rounded least-squares
    solution itself (the rounding of x alone is a relative perturbation of
    order 2^-53 per component), so whether the test ever fires is decided by
    rounding.  Everywhere else u = 2^-53.
  * LSQR-based SPIR solves each step's least-squares problem
    min ||r_i - A D^{-1} R^{-1} dy|| by LSQR from dy = 0, with the same two
    stopping rules applied to the LSQR update (phi_k / rho_k) w_k.
  * Column scaling (Alg. 4, first line) is on by default and is applied
    explicitly, A <- A diag(d)^{-1}; x is unscaled at the end (Alg. 4, last
    line).
"""
import ctypes
import math

import numpy as np

from . import _cbuild
from .philox import sparse_sign_matrix

U_ROUNDOFF = 2.0 ** -53
KW_STOP_U = 2.0 ** -52   # u of Alg. 4's step-2 test (Sec. 1.4's stated value)

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(_cbuild.build())
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        lib.or_householder_qr.argtypes = [i64, i64, dp, i64, dp]
        lib.or_apply_qt.argtypes = [i64, i64, dp, dp]
        lib.or_backsub.argtypes = [i64, dp, i64, dp, dp]
        lib.or_backsub_t.argtypes = [i64, dp, i64, dp, dp]
        lib.or_resid_dot2.argtypes = [i64, i64, dp, i64, dp, dp, dp, dp, dp]
        for f in (lib.or_householder_qr, lib.or_apply_qt, lib.or_backsub,
                  lib.or_backsub_t, lib.or_resid_dot2):
            f.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Dense building blocks
# ---------------------------------------------------------------------------

def householder_qr(M):
    """Householder QR of M (rows >= cols): Sec. 2.1 (sketch and QR) and Lemma 6.3
    (the analysis assumes Householder QR).

    Returns (R, V): R is the cols x cols upper-triangular factor and V the
    rows x cols matrix of unit reflector vectors (Q = H_0 H_1 ... with
    H_k = I - 2 v_k v_k^T).
    """
    W = np.array(M, dtype=np.float64, order="C", copy=True)
    rows, cols = W.shape
    if rows < cols:
        raise ValueError("householder_qr needs rows >= cols")
    V = np.empty((rows, cols), dtype=np.float64)
    _lib().or_householder_qr(rows, cols, _p(W), cols, _p(V))
    return np.ascontiguousarray(W[:cols, :cols]), V


def apply_qt(V, y):
    """Q^T y with the reflectors V returned by householder_qr."""
    out = _c64(y).copy()
    rows, cols = V.shape
    _lib().or_apply_qt(rows, cols, _p(_c64(V)), _p(out))
    return out


def backsub(R, y):
    """R^{-1} y by back substitution (Sec. 6, notation: triangular solves are
    computed by back substitution)."""
    R = _c64(R)
    n = R.shape[0]
    x = _c64(y).copy()
    _lib().or_backsub(n, _p(R), n, _p(x), _p(x))
    return x


def backsub_t(R, y):
    """R^{-T} y by forward substitution on R^T."""
    R = _c64(R)
    n = R.shape[0]
    x = _c64(y).copy()
    _lib().or_backsub_t(n, _p(R), n, _p(x), _p(x))
    return x


def qr_solve(A, b, return_R=False):
    """Least-squares solution of min ||b - A x|| (Sec. 1) by Householder QR:
    x = R^{-1} (Q^T b)[:n].  This is the classical direct solver the paper
    uses as its accuracy yardstick (Sec. 1, Fig. 1, Table 1)."""
    A = _c64(A)
    n = A.shape[1]
    R, V = householder_qr(A)
    y = apply_qt(V, b)[:n]
    x = backsub(R, y)
    return (x, R) if return_R else x


def qr_solve_lapack(A, b, return_R=False):
    """The least-squares solve of qr_solve, x = R^{-1} (Q^T b)[:n], with the
    factorisation and Q^T b taken from LAPACK's blocked Householder QR
    (dgeqrf / dormqr through scipy.linalg.qr_multiply: a library step) and
    the back substitution from this oracle.  For problems where the plain
    loops of householder_qr take minutes (m n^2 above ~1e11).  R may differ
    from householder_qr's by row signs; R^T R = A^T A either way, which is
    all kw_estimate needs of it."""
    import scipy.linalg as sl
    A = _c64(A)
    n = A.shape[1]
    qtb, R = sl.qr_multiply(A, _c64(b)[None, :], mode="right")
    R = np.ascontiguousarray(np.triu(R[:n, :n]))
    x = backsub(R, np.ascontiguousarray(qtb.ravel()[:n]))
    return (x, R) if return_R else x


def column_norms(A):
    """d_j = ||A[:, j]||_2 (Alg. 4, ColumnNorms)."""
    return np.sqrt(np.einsum("ij,ij->j", A, A))


def sketch(A, b, d, zeta, seed):
    """S [A b] with S the sparse sign embedding of Sec. 4.2 (Choice of
    embedding): S = zeta^{-1/2} [s_1 ... s_m].  The +-1 pattern is summed
    first and the factor zeta^{-1/2} applied once to the result."""
    m = A.shape[0]
    S = sparse_sign_matrix(m, d, zeta, seed)
    S = S.sign()  # the +-1 pattern
    c = 1.0 / math.sqrt(zeta)
    SA = np.asarray(S @ A) * c
    Sb = np.asarray(S @ b).ravel() * c
    return SA, Sb


def fixed_point_sketch(A, b, d, zeta, seed, row_chunks=None):
    """Unscaled S [A b] (the +-1 pattern of Sec. 4.2's sparse sign embedding,
    without the zeta^{-1/2} factor) summed in 64-bit fixed point per column,
    the summation order the CUDA library takes for large problems (the paper fixes
    none).  Every term a_ij is truncated toward zero to a multiple of 2^F_j,
    F_j = (E_j - 1022) + L - 63, where E_j is the largest biased exponent in
    column j over the rows summed (at least 1) and L the bit length of the
    longest source list (the most nonzeros in one row of S; at least 10).  The
    truncated terms are added exactly in integers, and each sum is rounded
    once to FP64 and scaled by 2^F_j.

    row_chunks: row boundaries [0, r_1, ..., m]; each chunk has its own E_j,
    and the chunk results are added in FP64 in chunk order.  Returns the
    (d, n + 1) array whose last column is S b.  Plain numpy and scipy integer
    arithmetic; the sparse product is a library step on exact integers.
    """
    import scipy.sparse as sp
    from .philox import sparse_sign_pattern
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    rows, signs = sparse_sign_pattern(m, d, zeta, seed)
    lmax = int(np.bincount(rows[rows >= 0].ravel(), minlength=d).max())
    L = 10
    while L < 40 and (1 << L) <= lmax:
        L += 1
    Ab = np.ascontiguousarray(np.concatenate([A, np.asarray(b, dtype=np.float64)[:, None]], axis=1))
    bounds = list(row_chunks) if row_chunks is not None else [0, m]
    out = None
    for c in range(len(bounds) - 1):
        r0, r1 = int(bounds[c]), int(bounds[c + 1])
        bits = Ab[r0:r1].view(np.uint64)
        e = ((bits >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
        E = np.maximum(e.max(axis=0), 1)
        F = (E - 1022) + L - 63
        shift = (1075 + F)[None, :] - e              # >= L - 10 >= 0 where e >= 1
        mant = (bits & np.uint64((1 << 52) - 1)) | np.uint64(1 << 52)
        keep = (e > 0) & (shift < 64)
        t = np.where(keep, mant >> np.minimum(shift, 63).astype(np.uint64), np.uint64(0))
        t = t.astype(np.int64)
        t = np.where((bits >> np.uint64(63)) == 1, -t, t)
        # sum over each row of S: the +-1 entries of S times the integer terms
        rr, ss = rows[r0:r1], signs[r0:r1]
        ok = rr >= 0
        cols = np.repeat(np.arange(r1 - r0, dtype=np.int64)[:, None], rr.shape[1], axis=1)
        S = sp.csr_matrix((ss[ok].astype(np.int64), (rr[ok], cols[ok])), shape=(d, r1 - r0),
                          dtype=np.int64)
        sums = np.asarray(S @ t, dtype=np.int64)
        part = sums.astype(np.float64) * np.ldexp(1.0, F)[None, :]
        out = part if out is None else out + part
    return out


def sigma_extremes(R):
    """(sigma_max, sigma_min) of R via the LAPACK SVD (a library step)."""
    s = np.linalg.svd(R, compute_uv=False)
    return float(s[0]), float(s[-1])


def q0_count(condest, eta, u=U_ROUNDOFF):
    """q0 of Theorem 7.1 (Sec. 7): max(1 + 2 log(1/(kappa u)) / log(1/(1.01 eta)), 11)."""
    e = 1.01 * eta
    if e <= 0.0:
        return 11.0
    val = 1.0 + 2.0 * math.log(1.0 / (condest * u)) / math.log(1.0 / e)
    return max(val, 11.0)


def step2_updates(condest, eta, max_inner=100):
    """Number of inner updates in the second refinement step: Alg. 5 with
    q = ceil(q0) produces dy_(q) after q - 1 updates."""
    q = int(math.ceil(q0_count(condest, eta)))
    return max(1, min(max_inner, q - 1))


# ---------------------------------------------------------------------------
# FOSSILS and SPIR
# ---------------------------------------------------------------------------

class _Problem:
    """Scaled problem data shared by FOSSILS and SPIR (Alg. 4 setup)."""

    def __init__(self, A, b, d, zeta, seed, eta, col_scale):
        A = _c64(A)
        b = _c64(b)
        self.m, self.n = A.shape
        self.d = int(d) if d else 12 * self.n
        self.zeta = zeta
        self.eta = eta if eta else math.sqrt(self.n / self.d)
        self.beta = self.eta ** 2
        self.alpha = (1.0 - self.beta) ** 2
        if col_scale:
            self.dcol = column_norms(A)
            self.As = A / self.dcol
        else:
            self.dcol = np.ones(self.n)
            self.As = A
        self.b = b
        self.SA, self.Sb = sketch(self.As, b, self.d, zeta, seed)
        self.R, V = householder_qr(self.SA)
        self.t = apply_qt(V, self.Sb)[: self.n]
        smax, smin = sigma_extremes(self.R)
        self.normest = smax
        self.condest = smax / smin if smin > 0 else math.inf

    def apply(self, z):
        """z -> R^{-T}(A^T(A(R^{-1} z))) in that order (Alg. 1; Sec. 6)."""
        w = backsub(self.R, z)
        return backsub_t(self.R, self.As.T @ (self.As @ w))

    def rhs(self, x):
        """c = R^{-T}(A^T(b - A x)) (Alg. 1, refinement right-hand side)."""
        r = self.b - self.As @ x
        return backsub_t(self.R, self.As.T @ r), r


def _polyak(P, c, alpha, beta, max_updates, thresh, check=None):
    """Polyak heavy ball on (R^{-T}A^T A R^{-1}) dy = c (Alg. 5 / Alg. 4 loop):
    dy = dy_old = c; Delta = alpha (c - M dy) + beta (dy - dy_old);
    (dy, dy_old) <- (dy + Delta, dy).  Stops after an update with
    ||Delta|| <= thresh when thresh is given, or when check(dy, k) (k updates
    done) returns True."""
    dy = c.copy()
    dy_old = c.copy()
    k = 0
    for _ in range(max_updates):
        delta = alpha * (c - P.apply(dy)) + beta * (dy - dy_old)
        dy_old = dy
        dy = dy + delta
        k += 1
        if thresh is not None and np.linalg.norm(delta) <= thresh:
            break
        if check is not None and check(dy, k):
            break
    return dy, k


def _cg(P, c, max_updates, thresh):
    """Conjugate gradient on M dy = c from dy = 0 (Alg. 3's inner solver)."""
    dy = np.zeros_like(c)
    res = c.copy()
    p = res.copy()
    rho = float(res @ res)
    k = 0
    for _ in range(max_updates):
        if rho == 0.0:
            break
        q = P.apply(p)
        gam = rho / float(p @ q)
        step = gam * p
        dy = dy + step
        res = res - gam * q
        rho_new = float(res @ res)
        p = res + (rho_new / rho) * p
        rho = rho_new
        k += 1
        if thresh is not None and np.linalg.norm(step) <= thresh:
            break
    return dy, k


def _lsqr(P, r, max_updates, thresh):
    """LSQR (Paige and Saunders) on min ||r - B dy||, B = A R^{-1} (the step's
    least-squares problem, eq. (ls-itref), right-preconditioned by R; Sec.
    "SPIR: Conjugate gradient or LSQR?"), from dy = 0.  Golub-Kahan
    bidiagonalisation of B started from r, plane rotations on the bidiagonal,
    and the update dy += (phi_k / rho_k) w_k, whose norm the stopping rule
    reads as SPIR reads CG's step."""
    def B(v):
        return P.As @ backsub(P.R, v)

    def BT(u):
        return backsub_t(P.R, P.As.T @ u)

    dy = np.zeros(P.n)
    beta = float(np.linalg.norm(r))
    if beta == 0.0:
        return dy, 0
    u = r / beta
    v = BT(u)
    alpha = float(np.linalg.norm(v))
    if alpha == 0.0:
        return dy, 0
    v = v / alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    k = 0
    for _ in range(max_updates):
        u = B(v) - alpha * u
        beta = float(np.linalg.norm(u))
        if beta > 0.0:
            u = u / beta
        v = BT(u) - beta * v
        alpha = float(np.linalg.norm(v))
        if alpha > 0.0:
            v = v / alpha
        rho = math.hypot(rhobar, beta)
        cs, sn = rhobar / rho, beta / rho
        theta = sn * alpha
        rhobar = -cs * alpha
        phi = cs * phibar
        phibar = sn * phibar
        step = (phi / rho) * w
        dy = dy + step
        w = v - (theta / rho) * w
        k += 1
        if thresh is not None and np.linalg.norm(step) <= thresh:
            break
        if alpha == 0.0 or phibar == 0.0:
            break
    return dy, k


def _solve(method, A, b, d, zeta, seed, eta, col_scale, max_inner, stop_gamma,
           stop_rho, n_refine, fixed_updates, kw_stop=False):
    P = _Problem(A, b, d, zeta, seed, eta, col_scale)
    x = backsub(P.R, P.t)  # sketch-and-solve x0 (Sec. 2.3)
    r0 = P.b - P.As @ x
    thresh1 = U_ROUNDOFF * (stop_gamma * P.normest * np.linalg.norm(x)
                            + stop_rho * P.condest * np.linalg.norm(r0))
    q2 = step2_updates(P.condest, P.eta, max_inner)
    xs = [x.copy()]
    cnorms = []
    iters = []
    for i in range(n_refine):
        c, r = P.rhs(x)
        cnorms.append(float(np.linalg.norm(c)))
        if fixed_updates is not None:
            nmax, th = fixed_updates, None
        elif i == 0:
            nmax, th = max_inner, thresh1
        else:
            nmax, th = q2, None
        check = None
        if kw_stop and i >= 1 and fixed_updates is None:
            # Alg. 4, second inner solve: every five updates (after updates
            # 1, 6, 11, ...) estimate the backward error of x + R^{-1} dy with
            # the sketched KW estimate (theta = ||A||_F / ||b||, on the column-
            # normalised A) and stop once it is below u ||A||_F, u = 2^-52.
            nmax = max_inner
            fro = float(np.linalg.norm(P.As))

            def check(dy_, k_, x_=x):
                if (k_ - 1) % 5 != 0:
                    return False
                xh = x_ + backsub(P.R, dy_)
                return sketched_kw(P.SA, P.As, P.b, xh) < KW_STOP_U * fro
        if method == "fossils":
            dy, k = _polyak(P, c, P.alpha, P.beta, nmax, th, check)
        elif method == "spir_lsqr":
            dy, k = _lsqr(P, r, nmax, th)
        else:
            dy, k = _cg(P, c, nmax, th)
        iters.append(k)
        x = x + backsub(P.R, dy)
        xs.append(x.copy())
    return {
        "x": x / P.dcol,
        "iterates": [v / P.dcol for v in xs],
        "iters": iters,
        "cnorms": cnorms,
        "condest": P.condest,
        "normest": P.normest,
        "thresh1": thresh1,
        "q2": q2,
        "alpha": P.alpha,
        "beta": P.beta,
        "d": P.d,
        "R": P.R,
        "dcol": P.dcol,
    }


def fossils(A, b, d=None, zeta=8, seed=0, eta=None, col_scale=True, max_inner=100,
            stop_gamma=10.0, stop_rho=0.4, n_refine=2, fixed_updates=None, kw_stop=False):
    """FOSSILS (Alg. 2 with the practical rules of Sec. 4.2 / Alg. 4, QR
    preconditioner): sketch, Householder QR, sketch-and-solve x0, then
    n_refine (default 2) refinement steps with the Polyak inner solver.
    kw_stop: end the second inner solve with Alg. 4's sketched
    Karlson-Walden test (every five updates, cap max_inner) instead of
    Theorem 7.1's count."""
    return _solve("fossils", A, b, d, zeta, seed, eta, col_scale, max_inner,
                  stop_gamma, stop_rho, n_refine, fixed_updates, kw_stop)


def spir(A, b, d=None, zeta=8, seed=0, eta=None, col_scale=True, max_inner=100,
         stop_gamma=10.0, stop_rho=0.4, n_refine=2, fixed_updates=None):
    """SPIR (Alg. 3): as FOSSILS with conjugate gradient as inner solver."""
    return _solve("spir", A, b, d, zeta, seed, eta, col_scale, max_inner,
                  stop_gamma, stop_rho, n_refine, fixed_updates)


def spir_lsqr(A, b, d=None, zeta=8, seed=0, eta=None, col_scale=True, max_inner=100,
              stop_gamma=10.0, stop_rho=0.4, n_refine=2, fixed_updates=None):
    """LSQR-based SPIR (Sec. "SPIR: Conjugate gradient or LSQR?"): as SPIR,
    with each refinement step's least-squares problem solved by LSQR with
    preconditioner R instead of CG on its normal equations; the same two
    stopping rules, applied to the LSQR step."""
    return _solve("spir_lsqr", A, b, d, zeta, seed, eta, col_scale, max_inner,
                  stop_gamma, stop_rho, n_refine, fixed_updates)


# ---------------------------------------------------------------------------
# Quality measures
# ---------------------------------------------------------------------------

def residual_dot2(A, b, x):
    """(r_hi, r_lo, g): r = b - A x and g = A^T r with compensated dot products."""
    A = _c64(A)
    m, n = A.shape
    x = _c64(x)
    r_hi = np.empty(m)
    r_lo = np.empty(m)
    g = np.empty(n)
    _lib().or_resid_dot2(m, n, _p(A), n, _p(_c64(b)), _p(x), _p(r_hi), _p(r_lo), _p(g))
    return r_hi, r_lo, g


def kw_estimate(A, b, xhat, theta=None, R_A=None):
    """Karlson-Walden estimate of the backward error (Sec. 4.1, the display
    defining BE-hat_theta):

        theta / sqrt(1 + theta^2 ||x||^2) *
            || (A^T A + lam I)^{-1/2} A^T r ||,
        lam = theta^2 ||r||^2 / (1 + theta^2 ||x||^2),  r = b - A x.

    theta defaults to ||A||_F / ||b|| (Sec. 4.2, "Adaptive stopping", item 2).
    (A^T A + lam I) = R_lam^T R_lam with R_lam the R factor of [R_A; sqrt(lam) I]
    (a QR of A makes the estimate O(mn), as Sec. 4.1 notes), so the norm is
    ||R_lam^{-T} A^T r||.  r and A^T r use compensated dot products.
    Returns the absolute estimate; divide by ||A||_F for the relative one.
    """
    A = _c64(A)
    b = _c64(b)
    xhat = _c64(xhat)
    n = A.shape[1]
    if theta is None:
        theta = np.linalg.norm(A) / np.linalg.norm(b)
    if R_A is None:
        R_A, _ = householder_qr(A)
    r_hi, r_lo, g = residual_dot2(A, b, xhat)
    nr = np.linalg.norm(r_hi)
    nx = np.linalg.norm(xhat)
    lam = theta ** 2 * nr ** 2 / (1.0 + theta ** 2 * nx ** 2)
    stacked = np.vstack([R_A, math.sqrt(lam) * np.eye(n)])
    R_lam, _ = householder_qr(stacked)
    y = backsub_t(R_lam, g)
    return theta / math.sqrt(1.0 + theta ** 2 * nx ** 2) * float(np.linalg.norm(y))


def sketched_kw(SA, A, b, xhat, theta=None):
    """Sketched Karlson-Walden estimate (Sec. 4.1, eq. (sketched-kw)):

        theta / sqrt(1 + theta^2 ||x||^2) *
            || ((SA)^T (SA) + lam I)^{-1/2} A^T r ||,
        lam = theta^2 ||r||^2 / (1 + theta^2 ||x||^2),  r = b - A x,

    evaluated as Alg. 4 does, through the SVD SA = U Sigma V^T:
    || (Sigma^2 + lam I)^{-1/2} V^T (A^T r) ||.  theta defaults to
    ||A||_F / ||b||.  r and A^T r use compensated dot products; the SVD is
    LAPACK's (a library step).  Returns the absolute estimate."""
    A = _c64(A)
    b = _c64(b)
    xhat = _c64(xhat)
    if theta is None:
        theta = np.linalg.norm(A) / np.linalg.norm(b)
    _, sig, Vt = np.linalg.svd(np.asarray(SA, dtype=np.float64), full_matrices=False)
    r_hi, _, g = residual_dot2(A, b, xhat)
    nr = np.linalg.norm(r_hi)
    nx = np.linalg.norm(xhat)
    lam = theta ** 2 * nr ** 2 / (1.0 + theta ** 2 * nx ** 2)
    y = (Vt @ g) / np.sqrt(sig ** 2 + lam)
    return theta / math.sqrt(1.0 + theta ** 2 * nx ** 2) * float(np.linalg.norm(y))


def kw_relative(A, b, xhat, R_A=None):
    """BE-hat_theta(x) / ||A||_F with theta = ||A||_F/||b|| (the target
    quantity of Sec. 4.2 item 2: backward stable when below ~u)."""
    return kw_estimate(A, b, xhat, R_A=R_A) / float(np.linalg.norm(A))


def forward_error(x, x_ref):
    return float(np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref))


def wedin_bound(kappa, normA, x, resid, u=U_ROUNDOFF):
    """First-order Wedin forward-error bound relative to ||x||:
    Fact 2.4 (Wedin) with eps = u, 2.23 kappa (||x|| + kappa ||r|| / ||A||) u / ||x||."""
    nx = float(np.linalg.norm(x))
    return 2.23 * kappa * (nx + kappa * resid / normA) * u / nx


# ---------------------------------------------------------------------------
# Complex problems (the Prony experiment, Sec. 5 "Runtime and iteration
# count" and the appendix on Prony's method: A in C^{m x n}, b in C^m)
# ---------------------------------------------------------------------------

def real_embedding(A):
    """The real 2m x 2n matrix of a complex m x n one, rows and columns
    interleaved:

        E[2i,   2k] = Re a_ik,   E[2i,   2k+1] = -Im a_ik,
        E[2i+1, 2k] = Im a_ik,   E[2i+1, 2k+1] =  Re a_ik,

    so that E [Re x_0, Im x_0, Re x_1, ...] is A x with its real and
    imaginary parts interleaved: ||E x_r|| = ||A x||, E^T E is the embedding
    of A^H A (each singular value of A twice), and the complex least-squares
    problem min ||b - A x|| is the real one min ||b_r - E x_r|| with b_r, x_r
    the interleaved parts.  ||E||_F = sqrt(2) ||A||_F."""
    A = np.asarray(A, dtype=np.complex128)
    m, n = A.shape
    E = np.empty((2 * m, 2 * n), dtype=np.float64)
    E[0::2, 0::2] = A.real
    E[0::2, 1::2] = -A.imag
    E[1::2, 0::2] = A.imag
    E[1::2, 1::2] = A.real
    return E


def as_real(v):
    """Interleaved real view [Re v_0, Im v_0, Re v_1, ...] of a complex vector."""
    return np.ascontiguousarray(np.asarray(v, dtype=np.complex128)).view(np.float64).copy()


def as_complex(v):
    """The complex vector of an interleaved real one."""
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64)).view(np.complex128).copy()


def solve_complex(method, A, b, **kw):
    """FOSSILS / SPIR / LSQR-SPIR of a complex problem: the real method on its
    real embedding (same solution), returning the complex x and the real
    method's result dict."""
    fn = {"fossils": fossils, "spir": spir, "spir_lsqr": spir_lsqr}[method]
    res = fn(real_embedding(A), as_real(b), **kw)
    return as_complex(res["x"]), res


def kw_relative_complex(A, b, xhat, R_E=None):
    """The Karlson-Walden estimate (Sec. 4.1) of a complex x relative to
    ||A||_F, theta = ||A||_F / ||b||, evaluated on the real embedding with
    that theta: the embedding keeps ||b||, ||x|| and ||r|| and maps A^H A and
    A^H r to E^T E and E^T r_r, so the norm in the estimate is the same
    number (||E||_F = sqrt(2) ||A||_F is why theta is passed).  R_E: the R
    factor of the embedding, if already computed."""
    A = np.asarray(A, dtype=np.complex128)
    nA = float(np.linalg.norm(A))
    theta = nA / float(np.linalg.norm(b))
    return kw_estimate(real_embedding(A), as_real(b), as_real(xhat), theta=theta,
                       R_A=R_E) / nA
