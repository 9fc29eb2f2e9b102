"""Plain definitions the Krylov sampler and the log-det estimator converge to.

* Section 4: x = Q^{-1/2} z, Q^{-1/2} the inverse of the principal square root,
  is a draw from N(0, Q^{-1}) when z ~ N(0, I).
* Section 1: the dense baseline Q = L L^T (Cholesky) gives
  log det Q = 2 sum_i log L_ii.
* Section 2: block-circulant Q is diagonalised by the FFT; the same holds for
  the cell-centred Neumann lattice with the DCT-II and for Dirichlet with the
  DST-I (constant kappa^2 only).
* Section 6: the Hutchinson terms v^T log(Q) v.
* Section 5.1: the linear solve x = Q^{-1} b of the sMMALA proposal mean.

Everything here is FP64.  Pins: tests/test_oracle_exact.py.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla

from . import stencil


# ---------------------------------------------------------------- dense (tiny n)
def dense_eigh(Q):
    """Eigen-decomposition of a (sparse or dense) SPD Q, ascending eigenvalues."""
    Qd = Q.toarray() if hasattr(Q, "toarray") else np.asarray(Q, dtype=np.float64)
    return np.linalg.eigh(Qd)


def matrix_function_dense(Q, Z, f):
    """f(Q) z for each row z of Z (rows are vectors), via dense eigh."""
    lam, U = dense_eigh(Q)
    Z = np.atleast_2d(np.asarray(Z, dtype=np.float64))
    return ((U * f(lam)) @ (U.T @ Z.T)).T


def sample_dense(Q, Z):
    """x = Q^{-1/2} z (Section 4) for each row z of Z, by dense eigh."""
    lam, _ = dense_eigh(Q)
    if lam[0] <= 0:
        raise ValueError("Q is not positive definite")
    return matrix_function_dense(Q, Z, lambda l: 1.0 / np.sqrt(l))


def logdet_cholesky(Q) -> float:
    """log det Q = 2 sum log L_ii with Q = L L^T (Section 1's factorisation)."""
    Qd = Q.toarray() if hasattr(Q, "toarray") else np.asarray(Q, dtype=np.float64)
    L = sla.cholesky(Qd, lower=True)
    return float(2.0 * np.sum(np.log(np.diag(L))))


def quadform_log_dense(Q, V) -> np.ndarray:
    """v^T log(Q) v for each row v of V (the Hutchinson summands, Section 6)."""
    lam, U = dense_eigh(Q)
    V = np.atleast_2d(np.asarray(V, dtype=np.float64))
    W = V @ U
    return (W * W) @ np.log(lam)


# ------------------------------------------------------ spectral (constant kappa)
def _fwd(bc, X):
    axes = tuple(range(X.ndim))
    if bc == "periodic":
        return sfft.fftn(X, axes=axes, norm="ortho")
    if bc == "neumann":
        return sfft.dctn(X, type=2, axes=axes, norm="ortho")
    if bc == "dirichlet":
        return sfft.dstn(X, type=1, axes=axes, norm="ortho")
    raise ValueError(bc)


def _inv(bc, X):
    axes = tuple(range(X.ndim))
    if bc == "periodic":
        return sfft.ifftn(X, axes=axes, norm="ortho").real
    if bc == "neumann":
        return sfft.idctn(X, type=2, axes=axes, norm="ortho")
    if bc == "dirichlet":
        return sfft.idstn(X, type=1, axes=axes, norm="ortho")
    raise ValueError(bc)


def spectral_apply(shape, bc, mu, v):
    """U diag(mu) U^T v where U is the lattice Laplacian's eigenbasis for ``bc``
    (unitary FFT / DCT-II / DST-I) and ``mu`` is given on the transform grid."""
    shape = tuple(int(s) for s in shape)
    X = np.asarray(v, dtype=np.float64).reshape(shape)
    return _inv(bc, np.asarray(mu) * _fwd(bc, X)).reshape(-1)


def spectral_coefficients(shape, bc, v):
    """Coefficients of v in the unitary eigenbasis (complex for periodic)."""
    shape = tuple(int(s) for s in shape)
    return _fwd(bc, np.asarray(v, dtype=np.float64).reshape(shape))


def sample_spectral(shape, bc, op, kappa2_const, tau, z, kappa2_prior=None):
    """x = Q^{-1/2} z for constant kappa^2 through the closed-form eigenvalues."""
    mu = stencil.operator_eigenvalues(shape, bc, op, kappa2_const, tau, kappa2_prior=kappa2_prior)
    return spectral_apply(shape, bc, 1.0 / np.sqrt(mu), z)


def logdet_spectral(shape, bc, op, kappa2_const, tau, kappa2_prior=None) -> float:
    """log det Q = sum of log eigenvalues (constant kappa^2)."""
    mu = stencil.operator_eigenvalues(shape, bc, op, kappa2_const, tau, kappa2_prior=kappa2_prior)
    return float(np.sum(np.log(mu)))


def quadform_log_spectral(shape, bc, op, kappa2_const, tau, V, kappa2_prior=None) -> np.ndarray:
    """v^T log(Q) v = sum_k |c_k|^2 log mu_k for each row v (constant kappa^2)."""
    mu = stencil.operator_eigenvalues(shape, bc, op, kappa2_const, tau, kappa2_prior=kappa2_prior)
    out = []
    for v in np.atleast_2d(V):
        c = spectral_coefficients(shape, bc, v)
        out.append(float(np.sum(np.abs(c) ** 2 * np.log(mu))))
    return np.array(out)


# ---------------------------------------------------------------- linear solves (Section 5.1)
def solve_sparse(Q, B):
    """x = Q^{-1} b for each row b of B (the sMMALA mean's system, Section 5.1),
    by a sparse LU factorisation of Q (SuperLU)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    lu = spla.splu(sp.csc_matrix(Q))
    return np.array([lu.solve(np.asarray(b, dtype=np.float64).reshape(-1)) for b in np.atleast_2d(B)])


def solve_spectral(shape, bc, op, kappa2_const, tau, b, kappa2_prior=None):
    """x = Q^{-1} b for constant kappa^2 through the closed-form eigenvalues."""
    mu = stencil.operator_eigenvalues(shape, bc, op, kappa2_const, tau, kappa2_prior=kappa2_prior)
    return spectral_apply(shape, bc, 1.0 / mu, b)


# ----------------------------------------------------- a second route to Q^{-1/2} z
def sample_stieltjes(Q, z, lam_lo, lam_hi, h=0.35, pad=30.0):
    """x = Q^{-1/2} z from the Stieltjes integral of the inverse square root,
    Q^{-1/2} = (2/pi) int_0^inf (Q + s^2 I)^{-1} ds = (2/pi) int_R e^u (Q + e^{2u} I)^{-1} du,
    by the trapezoid rule in u with step h on [log(lam_lo)/2 - pad, log(lam_hi)/2 + pad],
    one sparse LU solve per node.  [lam_lo, lam_hi] must contain the spectrum
    of Q (bounds suffice).  For an eigenvalue lam the integrand is
    sech(u - log(lam)/2) / (2 sqrt(lam)): the discretisation error is about
    4 exp(-pi^2 / h) relative and the truncation error about (2/pi) exp(-pad).
    A route independent of Algorithm 1, for variable-kappa^2 grids where no
    closed form exists."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    Qc = sp.csc_matrix(Q)
    n = Qc.shape[0]
    I = sp.identity(n, format="csc")
    z = np.asarray(z, dtype=np.float64).reshape(-1)
    lo = 0.5 * np.log(lam_lo) - pad
    hi = 0.5 * np.log(lam_hi) + pad
    nodes = int(np.ceil((hi - lo) / h))
    x = np.zeros(n)
    for k in range(nodes + 1):
        u = lo + k * h
        x += np.exp(u) * spla.splu(Qc + np.exp(2.0 * u) * I).solve(z)
    return (2.0 / np.pi) * h * x
