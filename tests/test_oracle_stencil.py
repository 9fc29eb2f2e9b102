"""Pins for oracle/stencil.py: operator assembly vs the per-cell neighbour
definition, closed-form spectra, and the Figure 3 matrix of Section 5.2."""
import os

import numpy as np
import pytest

from oracle import stencil

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("shape", [(5,), (3, 4), (4, 3), (2, 3, 4), (3, 3, 3)])
@pytest.mark.parametrize("bc", stencil.BCS)
@pytest.mark.parametrize("op", stencil.OPS)
def test_kronecker_assembly_matches_bruteforce(shape, bc, op):
    rng = np.random.default_rng(7)
    k2 = rng.uniform(0.1, 2.0, size=shape)
    # kappa2_prior is the prior's constant of spde_plus_diag (ignored by the other operators)
    Q = stencil.precision_matrix(shape, bc, op, k2, tau=1.7, kappa2_prior=0.6).toarray()
    Qb = stencil.precision_matrix_bruteforce(shape, bc, op, k2, tau=1.7, kappa2_prior=0.6)
    np.testing.assert_allclose(Q, Qb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Q, Q.T, atol=0)


@pytest.mark.parametrize("n", [1, 2, 3, 8, 9])
@pytest.mark.parametrize("bc", stencil.BCS)
def test_1d_closed_form_eigenpairs(n, bc):
    L = stencil.laplacian_1d(n, bc).toarray()
    lam, U = stencil.laplacian_eigen_1d(n, bc)
    np.testing.assert_allclose(U.T @ U, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(L @ U, U * lam, atol=1e-12)


@pytest.mark.parametrize("shape", [(4, 6), (3, 4, 5)])
@pytest.mark.parametrize("bc", stencil.BCS)
@pytest.mark.parametrize("op", stencil.OPS)
def test_lattice_eigenvalues_match_dense(shape, bc, op):
    Q = stencil.precision_matrix(shape, bc, op, 0.3, tau=2.0, kappa2_prior=0.6).toarray()
    lam = np.sort(stencil.operator_eigenvalues(shape, bc, op, 0.3, 2.0, kappa2_prior=0.6).reshape(-1))
    np.testing.assert_allclose(np.linalg.eigvalsh(Q), lam, rtol=1e-10, atol=1e-10)


def test_periodic_5pt_closed_form():
    # lambda_{jk} = kappa^2 + 4 - 2 cos(2 pi j / N) - 2 cos(2 pi k / N)
    N = 8
    Q = stencil.precision_matrix((N, N), "periodic", "shifted_laplacian", 0.1).toarray()
    j, k = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    lam = 0.1 + 4 - 2 * np.cos(2 * np.pi * j / N) - 2 * np.cos(2 * np.pi * k / N)
    np.testing.assert_allclose(np.linalg.eigvalsh(Q), np.sort(lam.reshape(-1)), atol=1e-12)


def _figure3_params():
    vals = {}
    with open(os.path.join(GOLDEN, "figure3_matrix.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                key, val = line.split()
                vals[key] = int(val)
    return vals


def test_figure3_matrix_structure():
    p = _figure3_params()
    side, scale, power = p["side"], p["scale"], p["power"]
    assert power == 2
    # the MATLAB gallery matrix: 4 on the diagonal, -1 to lattice neighbours
    n = side * side
    G = np.zeros((n, n))
    for y in range(side):
        for x in range(side):
            i = x + side * y
            G[i, i] = 4.0
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if 0 <= x + dx < side and 0 <= y + dy < side:
                    G[i, (x + dx) + side * (y + dy)] = -1.0
    Qm = (scale * G) @ (scale * G)
    Q = stencil.precision_matrix((side, side), "dirichlet", "spde_squared", 0.0, tau=scale ** 2)
    np.testing.assert_allclose(Q.toarray(), Qm, rtol=0, atol=1e-6)
    # 13-point stencil in the interior
    row = Q.getrow(15 + side * 15)
    assert row.nnz == 13
    # closed-form extreme eigenvalues: 31^4 (4 - 2cos(pi/31) - 2cos(pi/31))^2, ...
    h = np.pi / (side + 1)
    lmin = scale ** 2 * (4 - 4 * np.cos(h)) ** 2
    lmax = scale ** 2 * (4 - 4 * np.cos(side * h)) ** 2
    ev = np.linalg.eigvalsh(Qm)
    np.testing.assert_allclose([ev[0], ev[-1]], [lmin, lmax], rtol=1e-9)


@pytest.mark.parametrize("shape", [(5, 7, 9), (2, 3, 4), (6, 8), (3, 1, 5), (2, 2, 2)])
@pytest.mark.parametrize("bc", stencil.BCS)
@pytest.mark.parametrize("op", stencil.OPS)
def test_precision_rows_match_bruteforce(shape, bc, op):
    # sampled rows of Q (used for full-size checks) against the cell-by-cell assembly
    rng = np.random.default_rng(7)
    k = rng.uniform(0.1, 1.0, size=shape)
    n = int(np.prod(shape))
    rows = rng.choice(n, size=min(n, 9), replace=False)
    Qb = stencil.precision_matrix_bruteforce(shape, bc, op, k, tau=1.3, kappa2_prior=0.45)
    R = stencil.precision_rows(shape, bc, op, k, 1.3, rows, kappa2_prior=0.45).toarray()
    np.testing.assert_allclose(R, Qb[rows], rtol=0, atol=1e-12)


def test_spde_plus_diag_is_prior_plus_diagonal():
    # Q = tau ((kp + L)^2 + D): the spde_squared matrix with constant kp plus tau D
    shape = (5, 6)
    rng = np.random.default_rng(3)
    d = rng.uniform(0.0, 2.0, size=shape)
    d[1, 2] = 0.0
    for bc in stencil.BCS:
        Q = stencil.precision_matrix_bruteforce(shape, bc, "spde_plus_diag", d, tau=0.7, kappa2_prior=0.4)
        Qp = stencil.precision_matrix_bruteforce(shape, bc, "spde_squared", 0.4, tau=0.7)
        np.testing.assert_allclose(Q - Qp, 0.7 * np.diag(d.reshape(-1)), rtol=0, atol=1e-13)
