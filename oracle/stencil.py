"""Lattice precision matrices Q, assembled explicitly (oracle side).

Section 2 of the paper: the methods only need a cheap product Q v; for a GMRF
on a lattice Q is sparse and the product costs O(n).  The library's operator
family (its reading of the paper's lattice models, Sections 3 and 5):

* graph Laplacian L with unit spacing: (L v)_i = sum over lattice neighbours j
  of (v_i - v_j);
* boundary conditions: ``periodic`` (torus, Section 3), ``neumann``
  (cell-centred, a boundary cell only counts neighbours inside the grid) and
  ``dirichlet`` (values outside the grid are zero, so every cell has 2*dim on
  the diagonal);
* ``shifted_laplacian``: Q = tau (K + L), K = diag(kappa^2);
* ``spde_squared``:      Q = tau (K + L)^2  (a 13-point stencil in 2-D; the
  Figure 3 matrix (31^2 poisson(30))^2 of Section 5.2 is this operator with
  kappa^2 = 0, Dirichlet boundary, tau = 31^4);
* ``spde_plus_diag``:    Q = tau ((kp I + L)^2 + D), a stationary prior with
  constant ``kappa2_prior`` = kp plus the diagonal D = diag(kappa2) (the
  circulant-plus-diagonal precision of the sMMALA proposal, Sections 3 and
  5.1).

Grids are given slowest axis first: ``shape = (ny, nx)`` or ``(nz, ny, nx)``;
cell ``(z, y, x)`` has index ``x + nx*(y + ny*z)`` (C order).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

BCS = ("periodic", "neumann", "dirichlet")
OPS = ("shifted_laplacian", "spde_squared", "spde_plus_diag")


def laplacian_1d(n: int, bc: str) -> sp.csr_matrix:
    """1-D graph Laplacian on n points with boundary condition ``bc``."""
    if bc not in BCS:
        raise ValueError(bc)
    n = int(n)
    main = np.full(n, 2.0)
    off = -np.ones(n - 1)
    L = sp.diags([off, main, off], [-1, 0, 1], shape=(n, n), format="lil")
    if bc == "periodic":
        if n == 1:
            return sp.csr_matrix((1, 1))
        L[0, n - 1] += -1.0
        L[n - 1, 0] += -1.0
    elif bc == "neumann":
        L[0, 0] = 1.0 if n > 1 else 0.0
        L[n - 1, n - 1] = 1.0 if n > 1 else 0.0
    return sp.csr_matrix(L)


def laplacian(shape, bc: str) -> sp.csr_matrix:
    """Graph Laplacian of the lattice ``shape`` as a Kronecker sum of 1-D ones."""
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    L = sp.csr_matrix((n, n))
    for ax, s in enumerate(shape):
        left = int(np.prod(shape[:ax])) if ax > 0 else 1
        right = int(np.prod(shape[ax + 1:])) if ax + 1 < len(shape) else 1
        L = L + sp.kron(sp.kron(sp.identity(left), laplacian_1d(s, bc)), sp.identity(right))
    return sp.csr_matrix(L)


def _kappa_vector(shape, kappa2):
    n = int(np.prod(shape))
    k = np.asarray(kappa2, dtype=np.float64)
    if k.ndim == 0:
        return np.full(n, float(k))
    return k.reshape(n).astype(np.float64)


def precision_matrix(shape, bc: str, op: str, kappa2, tau: float = 1.0, kappa2_prior=None) -> sp.csr_matrix:
    """Q for the lattice operator family above (sparse, FP64)."""
    if op not in OPS:
        raise ValueError(op)
    if op == "spde_plus_diag":
        B = float(kappa2_prior) * sp.identity(int(np.prod(shape))) + laplacian(shape, bc)
        return sp.csr_matrix(float(tau) * (B @ B + sp.diags(_kappa_vector(shape, kappa2))))
    B = sp.diags(_kappa_vector(shape, kappa2)) + laplacian(shape, bc)
    Q = B if op == "shifted_laplacian" else B @ B
    return sp.csr_matrix(float(tau) * Q)


def _shifted_rows(shape, bc, kvec_at, rows):
    """Rows ``rows`` of B = K + L as a sparse (len(rows) x n) matrix, from the
    1-D Laplacians of each axis (row (c_0..c_{d-1}) of the Kronecker sum is the
    sum over axes of row c_ax of the 1-D matrix along that axis)."""
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    rows = np.asarray(rows, dtype=np.int64)
    strides = [int(np.prod(shape[ax + 1:])) for ax in range(len(shape))]
    coords = np.stack(np.unravel_index(rows, shape), axis=0)  # [dim][len]
    r_list, c_list, v_list = [np.arange(len(rows))], [rows], [kvec_at(rows)]
    for ax, s in enumerate(shape):
        L1 = laplacian_1d(s, bc).tocsr()
        for r, c in enumerate(coords[ax]):
            lo, hi = L1.indptr[c], L1.indptr[c + 1]
            cols1, vals1 = L1.indices[lo:hi], L1.data[lo:hi]
            base = rows[r] - c * strides[ax]
            r_list.append(np.full(len(cols1), r))
            c_list.append(base + cols1.astype(np.int64) * strides[ax])
            v_list.append(vals1)
    R = sp.csr_matrix((np.concatenate(v_list), (np.concatenate(r_list), np.concatenate(c_list))),
                      shape=(len(rows), n))
    R.sum_duplicates()
    return R


def precision_rows(shape, bc: str, op: str, kappa2, tau: float = 1.0, rows=(), kappa2_prior=None) -> sp.csr_matrix:
    """Rows ``rows`` of Q without assembling Q (for sampled checks of
    matrix-free products on grids too large to assemble)."""
    if op not in OPS:
        raise ValueError(op)
    shape = tuple(int(s) for s in shape)
    k = np.asarray(kappa2, dtype=np.float64)
    if k.ndim == 0:
        kvec_at = lambda idx: np.full(len(idx), float(k))  # noqa: E731
    else:
        kf = k.reshape(-1)
        kvec_at = lambda idx: kf[idx].astype(np.float64)  # noqa: E731
    if op == "spde_plus_diag":
        rows = np.asarray(rows, dtype=np.int64)
        kp_at = lambda idx: np.full(len(idx), float(kappa2_prior))  # noqa: E731
        R = _shifted_rows(shape, bc, kp_at, rows)
        cols = np.unique(R.indices)
        R = sp.csr_matrix(R[:, cols] @ _shifted_rows(shape, bc, kp_at, cols))
        n = int(np.prod(shape))
        D = sp.csr_matrix((kvec_at(rows), (np.arange(len(rows)), rows)), shape=(len(rows), n))
        return sp.csr_matrix(float(tau) * (R + D))
    R = _shifted_rows(shape, bc, kvec_at, rows)
    if op == "spde_squared":
        # rows of B B: (row_i of B) applied to the rows of B it touches
        cols = np.unique(R.indices)
        Rc = _shifted_rows(shape, bc, kvec_at, cols)
        R = sp.csr_matrix(R[:, cols] @ Rc)
    return sp.csr_matrix(float(tau) * R)


def precision_matrix_bruteforce(shape, bc: str, op: str, kappa2, tau: float = 1.0, kappa2_prior=None) -> np.ndarray:
    """Dense Q built cell by cell from the neighbour definition (pin for the above).

    Loops over every cell and every axis direction, adds the edge term
    (v_i - v_j) for each neighbour that exists under ``bc``; no Kronecker
    products.  Only for tiny grids.
    """
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    k = _kappa_vector(shape, kappa2)
    diag = None
    if op == "spde_plus_diag":
        diag, k = k, np.full(n, float(kappa2_prior))
    B = np.zeros((n, n))
    strides = [int(np.prod(shape[ax + 1:])) for ax in range(len(shape))]
    for idx in itertools.product(*[range(s) for s in shape]):
        i = sum(c * st for c, st in zip(idx, strides))
        B[i, i] += k[i]
        for ax in range(len(shape)):
            for step in (-1, 1):
                c = idx[ax] + step
                if 0 <= c < shape[ax]:
                    nb = list(idx)
                    nb[ax] = c
                elif bc == "periodic":
                    nb = list(idx)
                    nb[ax] = c % shape[ax]
                elif bc == "dirichlet":
                    B[i, i] += 1.0  # edge to a zero-valued ghost cell
                    continue
                else:  # neumann: no edge
                    continue
                j = sum(cc * st for cc, st in zip(nb, strides))
                B[i, i] += 1.0
                B[i, j] -= 1.0
    Q = B if op == "shifted_laplacian" else B @ B
    if diag is not None:
        Q = Q + np.diag(diag)
    return float(tau) * Q


def laplacian_eigen_1d(n: int, bc: str):
    """Closed-form eigenpairs of ``laplacian_1d`` (orthonormal eigenvectors as columns).

    periodic: 2 - 2 cos(2 pi k / n) with Fourier modes (real cos/sin basis);
    neumann:  2 - 2 cos(pi k / n), DCT-II vectors cos(pi k (i + 1/2) / n);
    dirichlet: 2 - 2 cos(pi k / (n + 1)), DST-I vectors sin(pi k (i + 1) / (n + 1)).
    """
    i = np.arange(n)
    if bc == "periodic":
        lam = []
        vecs = []
        for k in range(n):
            lam.append(2 - 2 * np.cos(2 * np.pi * k / n))
            if k == 0:
                vecs.append(np.ones(n))
            elif 2 * k == n:
                vecs.append(np.cos(np.pi * i))
            elif k < n - k:
                vecs.append(np.cos(2 * np.pi * k * i / n))
            else:
                vecs.append(np.sin(2 * np.pi * k * i / n))
        U = np.array(vecs).T
    elif bc == "neumann":
        k = np.arange(n)
        lam = 2 - 2 * np.cos(np.pi * k / n)
        U = np.cos(np.pi * np.outer(i + 0.5, k) / n)
    elif bc == "dirichlet":
        k = np.arange(1, n + 1)
        lam = 2 - 2 * np.cos(np.pi * k / (n + 1))
        U = np.sin(np.pi * np.outer(i + 1, k) / (n + 1))
    else:
        raise ValueError(bc)
    U = U / np.linalg.norm(U, axis=0)
    return np.asarray(lam, dtype=np.float64), U


def laplacian_eigenvalues(shape, bc: str) -> np.ndarray:
    """Eigenvalues of the lattice Laplacian on the tensor grid (array of ``shape``)."""
    lams = [laplacian_eigen_1d(s, bc)[0] for s in shape]
    grids = np.meshgrid(*lams, indexing="ij")
    return sum(grids)


def operator_eigenvalues(shape, bc: str, op: str, kappa2_const: float, tau: float = 1.0,
                         kappa2_prior=None) -> np.ndarray:
    """Eigenvalues of Q for a constant kappa^2 (array of ``shape``, same ordering
    as the spectral transforms in ``exact``).  For ``spde_plus_diag`` the
    constant diagonal is ``kappa2_const`` and the prior's constant
    ``kappa2_prior``."""
    if op == "spde_plus_diag":
        lam = float(kappa2_prior) + laplacian_eigenvalues(shape, bc)
        return float(tau) * (lam * lam + float(kappa2_const))
    lam = float(kappa2_const) + laplacian_eigenvalues(shape, bc)
    if op == "spde_squared":
        lam = lam * lam
    return float(tau) * lam
