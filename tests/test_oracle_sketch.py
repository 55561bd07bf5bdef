"""Pins for the oracle's random embedding (oracle/philox.py).

* Philox4x64-10 block function against numpy.random.Philox, an independent
  implementation of the same published generator (numpy advances its counter
  before producing a block, so its block k comes from counter k + 1).
* The rejection-sampling spec against a scalar per-row transcription of the
  same spec (the vectorised oracle must make the same choices).
* Structure of the sparse sign embedding (Sec. 4.2): zeta distinct rows per
  column, values +-zeta^{-1/2}, rows and signs roughly uniform.
* The sketch S [A b] against a dense S @ [A b].
* The embedding property of Fact 2.1 on a constructed problem.
"""
import math

import numpy as np
import pytest

from oracle import lsq_oracle as O
from oracle.philox import philox4x64_10, sparse_sign_matrix, sparse_sign_pattern
from lsq_problems import problem_svd


@pytest.mark.parametrize("key,ctr", [
    ((0, 0), (0, 0, 0, 0)),
    ((5, 7), (10, 0, 0, 0)),
    ((2 ** 64 - 1, 2 ** 63 + 11), (2 ** 64 - 2, 3, 2 ** 40, 99)),
    ((123456789, 987654321), (1, 2, 3, 4)),
])
def test_philox_matches_numpy(key, ctr):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(ctr, dtype=np.uint64))
    ref = bg.random_raw(8)
    big = sum(int(v) << (64 * i) for i, v in enumerate(ctr))
    for blk in range(2):
        nxt = (big + blk + 1) % (1 << 256)   # numpy's 256-bit counter increment
        cc = np.array([(nxt >> (64 * i)) & (2 ** 64 - 1) for i in range(4)], dtype=np.uint64)
        mine = philox4x64_10(cc.reshape(4, 1), np.array(key, dtype=np.uint64))[:, 0]
        assert np.array_equal(mine, ref[4 * blk: 4 * blk + 4])


def _pattern_scalar(j, d, zeta, seed):
    """Per-row transcription of the spec in oracle/philox.py."""
    key = np.array([seed, 0], dtype=np.uint64)
    rows, t, u = [], 0, []
    while len(rows) < zeta:
        w = philox4x64_10(np.array([[j], [t], [0], [0]], dtype=np.uint64), key)[:, 0]
        block = []
        for k in range(4):
            block += [int(w[k]) & 0xFFFFFFFF, int(w[k]) >> 32]
        u += block
        start = 1 if t == 0 else 0
        for v in block[start:]:
            if len(rows) == zeta:
                break
            h = (v * d) >> 32
            if h not in rows:
                rows.append(h)
        t += 1
    signs = [-1.0 if (u[0] >> k) & 1 else 1.0 for k in range(zeta)]
    return rows, signs


@pytest.mark.parametrize("d,zeta", [(600, 8), (10, 8), (8, 8), (37, 3), (5, 1)])
def test_pattern_matches_scalar_spec(d, zeta):
    m = 64
    rows, signs = sparse_sign_pattern(m, d, zeta, seed=17)
    for j in range(m):
        r, s = _pattern_scalar(j, d, zeta, 17)
        assert list(rows[j]) == r
        assert list(signs[j]) == s


def test_pattern_structure_and_uniformity():
    m, d, zeta = 200000, 600, 8
    rows, signs = sparse_sign_pattern(m, d, zeta, seed=3)
    srt = np.sort(rows, axis=1)
    assert (np.diff(srt, axis=1) > 0).all()          # distinct rows per column
    assert rows.min() >= 0 and rows.max() < d
    assert set(np.unique(signs)) == {-1.0, 1.0}
    counts = np.bincount(rows.ravel(), minlength=d)
    expect = m * zeta / d
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert chi2 < d + 6 * math.sqrt(2 * d)            # chi-square with d-1 dof
    frac_neg = float((signs < 0).mean())
    assert abs(frac_neg - 0.5) < 5 * 0.5 / math.sqrt(signs.size)


def test_sketch_matches_dense_product():
    rng = np.random.default_rng(0)
    m, n, d, zeta = 3000, 7, 84, 8
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    S = sparse_sign_matrix(m, d, zeta, seed=9).toarray()
    assert S.shape == (d, m)
    assert np.allclose(np.abs(S[S != 0]), 1 / math.sqrt(zeta), rtol=0, atol=1e-17)
    assert ((S != 0).sum(axis=0) == zeta).all()
    SA, Sb = O.sketch(A, b, d, zeta, seed=9)
    assert np.allclose(SA, S @ A, rtol=1e-14, atol=1e-13)
    assert np.allclose(Sb, S @ b, rtol=1e-14, atol=1e-13)


@pytest.mark.parametrize("m,n,d", [(4000, 50, 600), (4000, 50, 200)])
def test_embedding_whitens(m, n, d):
    """Fact 2.1: sigma(A R^{-1}) in [1/(1+eta), 1/(1-eta)], eta ~ sqrt(n/d)
    (Sec. 4.2; 1.25 sqrt(n/d) allows for the heuristic's slack)."""
    P = problem_svd(m, n, 1e8, 1e-6, seed=4)
    pr = O._Problem(P["A"], P["b"], d, 8, 11, None, True)
    s = np.linalg.svd(pr.As @ np.linalg.inv(pr.R), compute_uv=False)
    eta = 1.25 * math.sqrt(n / d)
    assert s.min() >= 1 / (1 + eta)
    assert s.max() <= 1 / (1 - eta)


def _brute_fixed_point(A, b, d, zeta, seed, bounds):
    """The fixed-point sketch from its definition with exact rationals: each
    term floor(|a| / 2^F_j) (signed), E_j from math.frexp, L the smallest
    L >= 10 with 2^L above the longest source list, integer sums rounded once
    to FP64 (Python float of an int), chunk results added in order."""
    from fractions import Fraction
    m, n = A.shape
    rows, signs = sparse_sign_pattern(m, d, zeta, seed)
    counts = [0] * d
    for i in range(m):
        for z in range(zeta):
            if rows[i, z] >= 0:
                counts[int(rows[i, z])] += 1
    L = 10
    while (1 << L) <= max(counts):
        L += 1
    cols = [A[:, j] for j in range(n)] + [b]
    out = [[None] * (n + 1) for _ in range(d)]
    for c in range(len(bounds) - 1):
        r0, r1 = bounds[c], bounds[c + 1]
        for j, col in enumerate(cols):
            E = 1
            for i in range(r0, r1):
                x = float(col[i])
                if x != 0.0:
                    E = max(E, math.frexp(x)[1] + 1022)
            F = (E - 1022) + L - 63
            q = Fraction(2) ** F
            sums = [0] * d
            for i in range(r0, r1):
                x = float(col[i])
                t = int(Fraction(abs(x)) / q)      # floor of a non-negative rational
                t = -t if x < 0 else t
                for z in range(zeta):
                    h = int(rows[i, z])
                    if h >= 0:
                        sums[h] += t if signs[i, z] > 0 else -t
            for h in range(d):
                v = math.ldexp(float(sums[h]), F)
                out[h][j] = v if out[h][j] is None else out[h][j] + v
    return np.array(out, dtype=np.float64)


@pytest.mark.parametrize("bounds", [[0, 300], [0, 101, 300], [0, 7, 150, 299, 300]])
def test_fixed_point_sketch_brute_force(bounds):
    """oracle.fixed_point_sketch equals the exact-rational brute force bit for
    bit, chunked or not, with signs, zeros and terms far below 2^F_j."""
    rng = np.random.default_rng(17)
    m, n, d, zeta, seed = 300, 5, 12, 3, 23
    A = rng.standard_normal((m, n)) * np.array([1.0, 1e-3, 1e5, 1.0, 3.0])
    A[::7, 0] = 0.0
    A[::11, 3] = 1e-30                       # below 2^F_3: truncated to 0
    b = rng.standard_normal(m) * 1e2
    got = O.fixed_point_sketch(A, b, d, zeta, seed, row_chunks=bounds)
    ref = _brute_fixed_point(A, b, d, zeta, seed, bounds)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


def test_fixed_point_sketch_close_to_exact_sum():
    """Each entry differs from the exact sum of S [A b] by less than the
    truncation of its terms (one 2^F_j per term) plus one rounding."""
    rng = np.random.default_rng(3)
    m, n, d, zeta, seed = 3000, 20, 60, 8, 5
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    got = O.fixed_point_sketch(A, b, d, zeta, seed)
    S = sparse_sign_matrix(m, d, zeta, seed).sign()
    ref = np.asarray(S @ np.concatenate([A, b[:, None]], axis=1))
    cnt = np.asarray(abs(S).sum(axis=1)).ravel()
    L = max(10, int(cnt.max()).bit_length())
    absmax = np.abs(np.concatenate([A, b[:, None]], axis=1)).max(axis=0)
    E = np.frexp(absmax)[1] + 1022
    step = np.ldexp(1.0, (E - 1022) + L - 63)
    absref = np.asarray(abs(S) @ np.abs(np.concatenate([A, b[:, None]], axis=1)))
    bound = cnt[:, None] * step[None, :] + 2.0 ** -52 * np.abs(ref) + 2 * cnt[:, None] * 2.0 ** -53 * absref
    assert (np.abs(got - ref) <= bound).all()
