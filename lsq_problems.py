"""Seeded synthetic least-squares problems shared by the tests, the bench and
the smoke check.

This module only builds inputs (A, b and the known solution); it holds none of
the solvers' arithmetic, so both the CUDA path and the CPU oracle can take
their inputs from it without sharing any method code.

Generators
----------
``problem_svd``  -- A = U diag(sigma) V^T with U (m x n) and V (n x n) the
    orthonormal factors of QR decompositions of seeded standard Gaussians
    (columns sign-fixed by sign(R_ii), which makes them Haar distributed),
    sigma log-spaced from 1 down to 1/kappa, x_true a standard Gaussian
    scaled to unit norm, and r a Gaussian projected (twice) onto the
    orthogonal complement of range(U) and scaled to the requested norm;
    b = A x_true + r.  This is the construction of the paper's Fig. 1 and
    Table 1 problems (Sec. 1: log-spaced singular values, Haar singular
    vectors, residual of a given norm orthogonal to range(A)).
``problem_gaussian`` -- A = (G / sqrt(m)) diag(sigma) V^T with G an m x n
    standard Gaussian, V Haar, sigma log-spaced 1..1/kappa, and
    b = A x_true + noise * g with x_true and g standard Gaussian.

Randomness: numpy's PCG64 Generator seeded by ``seed``; every draw happens
in a fixed order, so a (generator, shape, seed) triple always gives the
same problem on one machine.
"""
import numpy as np


def haar_orthonormal(rng, rows, cols):
    """Orthonormal rows x cols factor of a seeded Gaussian, columns sign-fixed."""
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s


def log_sigma(n, kappa):
    """n singular values 10^{p_i}, p_i equally spaced in [0, -log10(kappa)]."""
    if n == 1:
        return np.ones(1)
    return 10.0 ** (-np.linspace(0.0, np.log10(kappa), n))


def problem_svd(m, n, kappa, resid_norm, seed, keep_factors=True):
    """Constructed problem with known solution x_true (see module docstring)."""
    rng = np.random.default_rng(seed)
    U = haar_orthonormal(rng, m, n)
    V = haar_orthonormal(rng, n, n)
    sigma = log_sigma(n, kappa)
    A = np.ascontiguousarray((U * sigma) @ V.T)
    x = rng.standard_normal(n)
    x /= np.linalg.norm(x)
    g = rng.standard_normal(m)
    r = g - U @ (U.T @ g)
    r = r - U @ (U.T @ r)
    nr = np.linalg.norm(r)
    r = r * (resid_norm / nr) if nr > 0 else r
    b = A @ x + r
    out = {"A": A, "b": b, "x_true": x, "kappa": kappa, "resid_norm": resid_norm}
    if keep_factors:
        out.update({"U": U, "sigma": sigma, "V": V, "r_true": r})
    return out


def problem_gaussian(m, n, kappa, noise, seed, dtype=np.float64):
    """A = (G/sqrt(m)) diag(sigma) V^T, b = A x_true + noise * g."""
    rng = np.random.default_rng(seed)
    V = haar_orthonormal(rng, n, n)
    sigma = log_sigma(n, kappa)
    W = np.ascontiguousarray((sigma[:, None] * V.T) / np.sqrt(m))
    A = np.empty((m, n), dtype=np.float64)
    x = rng.standard_normal(n)
    b = np.empty(m)
    step = 65536
    for i0 in range(0, m, step):
        i1 = min(m, i0 + step)
        G = rng.standard_normal((i1 - i0, n))
        A[i0:i1] = G @ W
    g = rng.standard_normal(m)
    b[:] = A @ x + noise * g
    return {"A": A, "b": b, "x_true": x, "kappa": kappa, "noise": noise,
            "sigma": sigma, "V": V}


def problem_multi_rhs(m, n, k, kappa, noise, seed):
    """A built as in problem_svd (no residual), B = A X_true + noise * G (m x k)."""
    rng = np.random.default_rng(seed)
    U = haar_orthonormal(rng, m, n)
    V = haar_orthonormal(rng, n, n)
    sigma = log_sigma(n, kappa)
    A = np.ascontiguousarray((U * sigma) @ V.T)
    X = rng.standard_normal((n, k))
    B = np.ascontiguousarray(A @ X + noise * rng.standard_normal((m, k)))
    return {"A": A, "B": B, "X_true": X, "kappa": kappa, "noise": noise}


def problem_svd_torch(m, n, kappa, resid_norm, seed, device="cuda"):
    """problem_svd's construction generated with torch on `device` (seeded
    torch.Generator; factors from torch.linalg.qr), for sizes where host
    LAPACK would take minutes (m = 1e6, n = 1000).  Returns device tensors."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f64 = torch.float64

    def haar(rows, cols):
        q, r = torch.linalg.qr(torch.randn(rows, cols, generator=g, dtype=f64, device=device))
        s = torch.sign(torch.diagonal(r))
        s[s == 0] = 1.0
        return q * s

    U = haar(m, n)
    V = haar(n, n)
    sigma = torch.from_numpy(log_sigma(n, kappa)).to(device)
    A = ((U * sigma) @ V.T).contiguous()
    x = torch.randn(n, generator=g, dtype=f64, device=device)
    x /= torch.linalg.norm(x)
    gv = torch.randn(m, generator=g, dtype=f64, device=device)
    r = gv - U @ (U.T @ gv)
    r = r - U @ (U.T @ r)
    r *= resid_norm / torch.linalg.norm(r)
    b = A @ x + r
    del U
    return {"A": A, "b": b, "x_true": x, "kappa": kappa, "resid_norm": resid_norm}


def problem_multi_rhs_torch(m, n, k, kappa, noise, seed, device="cuda"):
    """problem_multi_rhs's construction with torch on `device` (for m = 2e6)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f64 = torch.float64

    def haar(rows, cols):
        q, r = torch.linalg.qr(torch.randn(rows, cols, generator=g, dtype=f64, device=device))
        s = torch.sign(torch.diagonal(r))
        s[s == 0] = 1.0
        return q * s

    U = haar(m, n)
    V = haar(n, n)
    sigma = torch.from_numpy(log_sigma(n, kappa)).to(device)
    A = ((U * sigma) @ V.T).contiguous()
    del U
    X = torch.randn(n, k, generator=g, dtype=f64, device=device)
    B = (A @ X + noise * torch.randn(m, k, generator=g, dtype=f64, device=device)).contiguous()
    return {"A": A, "B": B, "X_true": X, "kappa": kappa, "noise": noise}


def problem_prony(m, n, seed, noise=1e-6, dt=0.25, spread=3.0):
    """The first least-squares problem of Prony's method (the paper's appendix
    on Prony's method, its algorithm's first line), synthetic: measurements
    f_j = sum_i mu_i z_i^j + eps_j for 0 <= j <= m + n - 1 with
    z_i = exp(-1j dt lambda_i) on the unit circle, lambda_i uniform in
    [-spread, spread], mu_i > 0 summing to 1, eps_j complex Gaussian with
    standard deviation `noise` (the paper: 1e-6).  A[i, j] = f[n - 1 + i - j],
    b[i] = f[n + i] (0-based), so A is Toeplitz, and with noise-free data b
    lies in range(A) (the linear-prediction equations); x_true = None."""
    rng = np.random.default_rng(seed)
    lam = np.sort(rng.uniform(-spread, spread, n))
    z = np.exp(-1j * dt * lam)
    mu = rng.dirichlet(np.ones(n))
    j = np.arange(m + n)
    f = (mu[None, :] * np.exp(-1j * dt * np.outer(j, lam))).sum(axis=1)
    eps = rng.standard_normal(m + n) + 1j * rng.standard_normal(m + n)
    f = f + noise / np.sqrt(2.0) * eps
    idx = (n - 1) + np.arange(m)[:, None] - np.arange(n)[None, :]
    A = np.ascontiguousarray(f[idx])
    b = np.ascontiguousarray(f[n + np.arange(m)])
    return {"A": A, "b": b, "z": z, "mu": mu, "lam": lam}


def problem_sparse(m, n, k, seed, delta=None, noise=1e-6):
    """Sparse A in CSR form, a synthetic stand-in for the paper's SuiteSparse
    matrices.  Each row holds k entries (k even, n even) in k / 2 column
    pairs (2q, 2q + 1): the q of a row run through an arithmetic progression
    modulo n / 2 with a random start and a random step coprime to n / 2, so
    they are distinct.  A pair's values are (a, a (1 + delta xi)) with a, xi
    standard normal (nearly dependent columns, condition ~ 1 / delta), or two
    independent normals when delta is None.  Columns are then scaled by
    10^U(-2, 2).  b = A x_true + noise g with x_true, g standard normal
    (x_true over sqrt(n)).  Returns row_ptr (int64, m + 1), col (int32),
    val (float64), b, x_true and the column scales."""
    import math
    rng = np.random.default_rng(seed)
    assert k % 2 == 0 and n % 2 == 0 and k // 2 <= n // 2
    h = n // 2
    units = np.array([g for g in range(1, h + 1) if math.gcd(g, h) == 1], dtype=np.int64)
    start = rng.integers(0, h, m)
    step = units[rng.integers(0, len(units), m)]
    q = (start[:, None] + np.arange(k // 2)[None, :] * step[:, None]) % h
    q = np.sort(q, axis=1)
    col = np.empty((m, k), dtype=np.int32)
    col[:, 0::2] = 2 * q
    col[:, 1::2] = 2 * q + 1
    a = rng.standard_normal((m, k // 2))
    val = np.empty((m, k))
    val[:, 0::2] = a
    if delta is None:
        val[:, 1::2] = rng.standard_normal((m, k // 2))
    else:
        val[:, 1::2] = a * (1.0 + delta * rng.standard_normal((m, k // 2)))
    scale = 10.0 ** rng.uniform(-2, 2, n)
    val = val * scale[col]
    row_ptr = np.arange(m + 1, dtype=np.int64) * k
    col = col.ravel()
    val = val.ravel()
    x_true = rng.standard_normal(n) / np.sqrt(n)
    Ax = (val.reshape(m, k) * x_true[col.reshape(m, k)]).sum(axis=1)
    b = Ax + noise * rng.standard_normal(m)
    return {"row_ptr": row_ptr, "col": col, "val": val, "b": b, "x_true": x_true,
            "scale": scale}


def csr_to_dense(P, m, n):
    """The dense m x n matrix of problem_sparse's CSR arrays."""
    A = np.zeros((m, n))
    rows = np.repeat(np.arange(m), np.diff(P["row_ptr"]))
    A[rows, P["col"]] = P["val"]
    return A
