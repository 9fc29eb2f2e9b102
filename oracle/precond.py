"""Constant-coefficient preconditioner M = F F^T (Proposition 1, Section 5).

Proposition 1: if u ~ N(0, (F^{-1} Q F^{-T})^{-1}) then F^T x = u gives x with
precision Q.  Section 5.1 / Theorem 2 use the (block) circulant prior as M; the
build takes M to be the same lattice operator as Q with kappa^2 replaced by a
constant kappa_bar^2 and with a boundary condition ``kind`` whose Laplacian is
diagonalised by a fast transform:

* ``periodic``  -- the circulant version on the grid's own torus (FFT);
* ``neumann``   -- the circulant version on the mirror-extended (2N)^d torus,
  restricted to mirror-symmetric vectors, i.e. the cell-centred Neumann
  operator (DCT-II);
* ``dirichlet`` -- the odd-extension analogue (DST-I).

F is the symmetric square root M^{1/2} (so F^T = F), hence
x = M^{-1/2} u and A = F^{-1} Q F^{-T} = M^{-1/2} Q M^{-1/2}.
Section 6.2: log det Q = log det A + log det M (the paper prints the second
term with a minus sign; det(F^{-1} Q F^{-T}) = det Q / det(F)^2 fixes it as
plus, and tests/test_oracle_lanczos.py pins the sign densely).
"""
from __future__ import annotations

import numpy as np

from . import exact, stencil


def kappa2_bar(kappa2) -> float:
    """Default constant for M: the geometric mean exp(mean log kappa^2)."""
    k = np.asarray(kappa2, dtype=np.float64)
    return float(np.exp(np.mean(np.log(k))))


def symbol(shape, kind, op, kbar2, tau):
    """Eigenvalues mu of M on the transform grid of ``kind``."""
    return stencil.operator_eigenvalues(shape, kind, op, kbar2, tau)


def apply_power(shape, kind, op, kbar2, tau, v, power):
    """M^power v through the closed-form spectrum."""
    mu = symbol(shape, kind, op, kbar2, tau)
    return exact.spectral_apply(shape, kind, mu ** power, v)


def logdet(shape, kind, op, kbar2, tau) -> float:
    """log det M = sum log mu."""
    return float(np.sum(np.log(symbol(shape, kind, op, kbar2, tau))))


def matrix(shape, kind, op, kbar2, tau):
    """M itself as a sparse matrix (the same operator family with constant kappa^2)."""
    return stencil.precision_matrix(shape, kind, op, kbar2, tau)


def dense_inv_sqrt(shape, kind, op, kbar2, tau):
    """Dense M^{-1/2} (tiny grids), by applying the spectral map to the identity."""
    n = int(np.prod(shape))
    cols = [apply_power(shape, kind, op, kbar2, tau, e, -0.5) for e in np.identity(n)]
    return np.array(cols).T


def preconditioned_operator_dense(Q, shape, kind, op, kbar2, tau):
    """Dense A = M^{-1/2} Q M^{-1/2} (tiny grids)."""
    P = dense_inv_sqrt(shape, kind, op, kbar2, tau)
    Qd = Q.toarray() if hasattr(Q, "toarray") else np.asarray(Q)
    A = P @ Qd @ P
    return 0.5 * (A + A.T), P


def sample_prop1_dense(Q, shape, kind, op, kbar2, tau, Z):
    """Exact Proposition 1 map x = M^{-1/2} (M^{-1/2} Q M^{-1/2})^{-1/2} z."""
    A, P = preconditioned_operator_dense(Q, shape, kind, op, kbar2, tau)
    U = exact.sample_dense(A, Z)
    return (P @ np.atleast_2d(U).T).T
