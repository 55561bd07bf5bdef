"""CPU FP64 oracle for the FOSSILS / SPIR least-squares hot path.

TEST INFRASTRUCTURE ONLY.  This package is the independent reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg (``--impl reference`` and the
``cpu_baseline`` object) may import, call, link or execute anything here.  It
shares no code, header, table or constant generator with the CUDA path and
never calls it; the product path fails loudly when its CUDA library is
missing instead of falling back to this package.

Modules
-------
philox      Philox4x64-10 and the sparse sign embedding spec (Sec. 4.2).
lsq_oracle  Householder QR solve, sketch, FOSSILS (Alg. 2 / Alg. 4), SPIR
            (Alg. 3), the Karlson-Walden estimate (Sec. 4.1), q0 (Theorem 7.1),
            complex problems through their real embedding.
liboracle.c plain C loops for the QR, triangular solves and compensated
            residuals, built by _cbuild.build().

Pins (tests marked "not gpu"): Philox against numpy's Philox; the sketch
against a dense S @ A; the QR against LAPACK and an extended-precision
normal-equations solve on tiny inputs; triangular solves against SciPy; the
Karlson-Walden estimate against its closed form in a known SVD basis
(App. A.1, proof of Theorem 2.8, generalised to theta); the Polyak solver
against the identity-sketch special case and the exact-arithmetic
contraction bound of the Polyak-with-noise lemma (Sec. 7.1); CG against finite termination; FOSSILS/SPIR against the paper's
printed numbers (Table 1, Table 2) and the known solutions of constructed
problems.  Parity of the exact backward error itself is unpinned: its
formula is not in the paper.
"""
from . import lsq_oracle, philox  # noqa: F401
from .lsq_oracle import (  # noqa: F401
    U_ROUNDOFF, apply_qt, backsub, backsub_t, column_norms, fixed_point_sketch, forward_error, fossils,
    householder_qr, kw_estimate, kw_relative, q0_count, qr_solve, qr_solve_lapack, residual_dot2,
    sigma_extremes, sketch, sketched_kw, spir, spir_lsqr, step2_updates, wedin_bound,
    real_embedding, as_real, as_complex, solve_complex, kw_relative_complex)
