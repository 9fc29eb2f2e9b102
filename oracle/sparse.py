"""General sparse precision matrices with an incomplete-Cholesky factor as the
preconditioner (Section 5.2, Figure 3; Proposition 1 with F the factor).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and the CPU legs of
``bench.py``, never by the product path (see ``oracle/__init__.py``).

Section 5.2 proposes the incomplete Cholesky factorisation of Q as a generic
preconditioner: M = F F^T with F lower triangular, sparse, F F^T close to Q.
Proposition 1 then gives a sample as x = F^{-T} A^{-1/2} z with
A = F^{-1} Q F^{-T}, and Section 6 the log-determinant as
log det Q = log det A + 2 sum_i log F_ii.  The paper compares factors with
several drop thresholds but states no dropping rule; the reading used here
(and by the library) is a left-looking threshold rule that does not depend on
the scale of Q (the updated entry is compared with the column norm of A' in
the same units):

  for column j = 0 .. n-1 of A' = Q + shift diag(Q):
      w      = A'[j:, j] - F[j:, :j] F[j, :j]^T
      F_jj   = sqrt(w_0)               (w_0 <= 0: breakdown, Q not factorable)
      F_ij   = w_i / F_jj  for i > j, kept unless
               IC(0)  (droptol None): A'_ij == 0   (no fill outside Q's pattern)
               ICT    (droptol >= 0): |w_i| < droptol * ||A'[j:, j]||_1

droptol = 0 keeps every entry (the exact Cholesky factor); droptol = inf keeps
only the diagonal (F = diag(A')^{1/2}, a Jacobi preconditioner).

Everything here is dense FP64 (numpy / scipy.linalg), for n up to a few
thousand: obviously correct rather than fast.

Pins (tests/test_oracle_sparse.py):
  ``ichol``          droptol 0 equals ``numpy.linalg.cholesky``; IC(0) on a
                     tridiagonal matrix is exact; F F^T equals A' on the kept
                     pattern, and each dropped entry's update is below its
                     threshold (checked from F and A' alone); droptol inf is
                     Jacobi.
  ``precond_map``    S S^T = Q^{-1} for S = F^{-T} A^{-1/2}; with the exact
                     Cholesky factor A = I and x = F^{-T} z.
  ``logdet_precond`` equals the dense Cholesky log-determinant.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


class NotFactorable(ValueError):
    """A non-positive pivot in the incomplete factorisation."""


def csr(rowptr, colind, val, n=None) -> sp.csr_matrix:
    """CSR arrays -> scipy matrix (no arithmetic)."""
    n = len(rowptr) - 1 if n is None else n
    return sp.csr_matrix((np.asarray(val, dtype=np.float64), np.asarray(colind), np.asarray(rowptr)), shape=(n, n))


def ichol(Q, droptol=None, shift=0.0) -> sp.csr_matrix:
    """Lower-triangular incomplete Cholesky factor F of Q + shift diag(Q)
    (Section 5.2), by the column rule in the module notes.  droptol None:
    IC(0); droptol >= 0: threshold dropping.  Raises NotFactorable."""
    A = Q.toarray() if sp.issparse(Q) else np.array(Q, dtype=np.float64)
    A = A + shift * np.diag(np.diag(A))
    n = A.shape[0]
    F = np.zeros((n, n))
    for j in range(n):
        w = A[j:, j] - F[j:, :j] @ F[j, :j]
        if not w[0] > 0.0:
            raise NotFactorable("pivot %d is %g" % (j, w[0]))
        d = np.sqrt(w[0])
        col = w[1:] / d
        if droptol is None:
            col[A[j + 1:, j] == 0.0] = 0.0
        else:
            col[np.abs(w[1:]) < droptol * np.abs(A[j:, j]).sum()] = 0.0
        F[j, j] = d
        F[j + 1:, j] = col
    return sp.csr_matrix(F)


def preconditioned_matrix(Q, F) -> np.ndarray:
    """A = F^{-1} Q F^{-T} (dense, symmetrised)."""
    Fd = F.toarray() if sp.issparse(F) else np.asarray(F)
    Qd = Q.toarray() if sp.issparse(Q) else np.asarray(Q)
    X = sla.solve_triangular(Fd, Qd, lower=True)       # F^{-1} Q
    A = sla.solve_triangular(Fd, X.T, lower=True)      # F^{-1} (F^{-1} Q)^T = F^{-1} Q F^{-T}
    return 0.5 * (A + A.T)


def precond_map(Q, F):
    """(lam, U, Fd): eigenpairs of A = F^{-1} Q F^{-T} and the dense factor, so
    that S = F^{-T} U diag(lam^{-1/2}) U^T is the sampling map of Proposition 1."""
    lam, U = np.linalg.eigh(preconditioned_matrix(Q, F))
    return lam, U, (F.toarray() if sp.issparse(F) else np.asarray(F))


def sample_precond_dense(Q, F, Z) -> np.ndarray:
    """x = F^{-T} A^{-1/2} z for each row z of Z ([nvec][n])."""
    lam, U, Fd = precond_map(Q, F)
    Z = np.atleast_2d(np.asarray(Z, dtype=np.float64))
    Y = (U @ ((U.T @ Z.T) / np.sqrt(lam)[:, None]))   # A^{-1/2} z, column per vector
    return sla.solve_triangular(Fd.T, Y, lower=False).T


def quadform_log_precond(Q, F, V) -> np.ndarray:
    """q_i = v_i^T log(A) v_i for each row v_i of V (the quadrature targets of
    the preconditioned Hutchinson estimator, Section 6)."""
    lam, U, _ = precond_map(Q, F)
    C = U.T @ np.atleast_2d(np.asarray(V, dtype=np.float64)).T
    return (np.log(lam)[:, None] * C * C).sum(axis=0)


def logdet_factor(F) -> float:
    """log det (F F^T) = 2 sum_i log F_ii."""
    return 2.0 * float(np.log(F.diagonal()).sum())


def logdet_precond(Q, F) -> float:
    """log det Q = log det A + log det(F F^T)  (Section 6.2 with M = F F^T)."""
    lam, _, _ = precond_map(Q, F)
    return float(np.log(lam).sum()) + logdet_factor(F)


def apply_lower_inv(F, V) -> np.ndarray:
    """F^{-1} v for each row v of V."""
    Fd = F.toarray() if sp.issparse(F) else np.asarray(F)
    return sla.solve_triangular(Fd, np.atleast_2d(V).T, lower=True).T


def apply_upper_inv(F, V) -> np.ndarray:
    """F^{-T} v for each row v of V."""
    Fd = F.toarray() if sp.issparse(F) else np.asarray(F)
    return sla.solve_triangular(Fd.T, np.atleast_2d(V).T, lower=False).T
