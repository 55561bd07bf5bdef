"""Oracle: counter-based random numbers and the sparse sign embedding.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import this module;
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg use it.

What it follows
---------------
* Sparse sign embedding (Sec. 4.2, "Choice of embedding"): S = zeta^{-1/2}
  [s_1 ... s_m], each column s_j (it lives in R^d) holding zeta nonzeros equal
  to +-1 with equal probability, at uniformly random distinct rows.
* The paper only says "uniformly random".  This project fixes one concrete,
  reproducible spec so that the CUDA sketch and this oracle build the same S
  independently:

  - generator: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), written
    here from its published round function;
  - for column j of S (row j of A): counter = (j, t, 0, 0) for
    t = 0, 1, 2, ...; key = (seed, 0);
  - every block gives four 64-bit words W0..W3; each word is split into two
    32-bit halves (low half first), giving the stream u_0, u_1, u_2, ...;
  - u_0 holds the signs: the k-th accepted nonzero is -1 iff bit k of u_0 is
    set (so zeta <= 32);
  - u_1, u_2, ... are candidate rows h = floor(u * d / 2^32); a candidate is
    accepted unless it equals an earlier accepted row of the same column;
    stop once zeta rows are accepted (sampling without replacement).

Pins (tests/test_oracle_sketch.py): the Philox block function is checked
against ``numpy.random.Philox`` (an independent implementation of the same
published generator); the embedding's structure (zeta distinct rows per
column, values +-zeta^{-1/2}) and the sketch product against a dense S @ A.
"""
import numpy as np

_M0 = np.uint64(0xD2E7470EE14C6C93)
_M1 = np.uint64(0xCA5A826395121157)
_W0 = np.uint64(0x9E3779B97F4A7C15)
_W1 = np.uint64(0xBB67AE8584CAA73B)
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo64(a, b):
    """Full 64x64 -> 128-bit product of uint64 arrays, returned as (hi, lo)."""
    a0 = a & _MASK32
    a1 = a >> _S32
    b0 = b & _MASK32
    b1 = b >> _S32
    p00 = a0 * b0
    p01 = a0 * b1
    p10 = a1 * b0
    p11 = a1 * b1
    mid = (p00 >> _S32) + (p01 & _MASK32) + (p10 & _MASK32)
    hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
    lo = a * b  # wraps modulo 2^64
    return hi, lo


def philox4x64_10(ctr, key):
    """Philox4x64 with 10 rounds.

    ctr: (4, N) uint64 array of counters; key: (2, N) or (2,) uint64 keys.
    Returns a (4, N) uint64 array.  Ten rounds, with the key bumped by the
    Weyl constants between rounds (Salmon et al., SC'11, Sec. 5).
    """
    with np.errstate(over="ignore"):
        c0, c1, c2, c3 = (np.array(ctr[i], dtype=np.uint64) for i in range(4))
        k0 = np.array(key[0], dtype=np.uint64)
        k1 = np.array(key[1], dtype=np.uint64)
        for r in range(10):
            if r > 0:
                k0 = k0 + _W0
                k1 = k1 + _W1
            hi0, lo0 = _mulhilo64(_M0, c0)
            hi1, lo1 = _mulhilo64(_M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3])


def _stream_block(rows, t, seed):
    """32-bit stream values u_{8t..8t+7} for the given A-rows (Philox block t)."""
    n = rows.shape[0]
    ctr = np.zeros((4, n), dtype=np.uint64)
    ctr[0] = rows.astype(np.uint64)
    ctr[1] = np.uint64(t)
    key = np.array([np.uint64(seed), np.uint64(0)], dtype=np.uint64)
    w = philox4x64_10(ctr, key)
    out = np.empty((n, 8), dtype=np.uint64)
    for k in range(4):
        out[:, 2 * k] = w[k] & _MASK32
        out[:, 2 * k + 1] = w[k] >> _S32
    return out


def sparse_sign_pattern(m, d, zeta, seed):
    """Rows and signs of the sparse sign embedding S (d x m).

    Returns (rows, signs): rows is an (m, zeta) int64 array, rows[j, k] is the
    row of S holding the k-th nonzero of column j; signs is (m, zeta) float64
    with entries +-1.  The nonzero value itself is signs * zeta^{-1/2}.
    """
    if not (1 <= zeta <= 32 and zeta <= d):
        raise ValueError("need 1 <= zeta <= min(d, 32)")
    js = np.arange(m, dtype=np.int64)
    rows = np.full((m, zeta), -1, dtype=np.int64)
    count = np.zeros(m, dtype=np.int64)
    sign_word = None
    t = 0
    pending = js
    while pending.size:
        u = _stream_block(pending, t, seed)
        start = 0
        if t == 0:
            sign_word = u[:, 0].copy()
            start = 1
        for q in range(start, 8):
            h = ((u[:, q] * np.uint64(d)) >> _S32).astype(np.int64)
            cur = rows[pending]
            need = count[pending] < zeta
            dup = (cur == h[:, None]).any(axis=1)
            take = need & ~dup
            idx = pending[take]
            rows[idx, count[idx]] = h[take]
            count[idx] += 1
        pending = pending[count[pending] < zeta]
        t += 1
    bits = (sign_word[:, None] >> np.arange(zeta, dtype=np.uint64)[None, :]) & np.uint64(1)
    signs = np.where(bits == 1, -1.0, 1.0)
    return rows, signs


def sparse_sign_matrix(m, d, zeta, seed):
    """S as a scipy CSR matrix (d x m) with nonzeros +-zeta^{-1/2}."""
    import scipy.sparse as sp
    rows, signs = sparse_sign_pattern(m, d, zeta, seed)
    cols = np.repeat(np.arange(m, dtype=np.int64), zeta)
    vals = (signs * (1.0 / np.sqrt(zeta))).ravel()
    return sp.csr_matrix((vals, (rows.ravel(), cols)), shape=(d, m))
