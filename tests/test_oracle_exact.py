"""Pins for oracle/exact.py: Q^{-1/2} z and log det Q by two independent routes
(dense eigh / Cholesky vs closed-form spectral transforms) and by the defining
identities."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import exact, stencil
from paper_1312_1476_gb300 import inputs

SHAPES = [(6, 8), (5, 7), (3, 4, 5)]
KP = 0.45  # the prior's constant of spde_plus_diag (ignored by the other operators)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", stencil.BCS)
@pytest.mark.parametrize("op", stencil.OPS)
def test_dense_sample_is_principal_inverse_sqrt(shape, bc, op):
    rng = np.random.default_rng(3)
    k2 = rng.uniform(0.05, 1.0, size=shape)
    Q = stencil.precision_matrix(shape, bc, op, k2, tau=1.3, kappa2_prior=KP)
    z = inputs.gaussian_vectors(2, int(np.prod(shape)), seed=5, dtype=np.float64)
    x = exact.sample_dense(Q, z)
    for xi, zi in zip(x, z):
        # x^T Q x = ||z||^2 and Q (Q^{-1/2} (Q^{-1/2} z)) = z (sparse matvec, no eigh)
        assert abs(xi @ (Q @ xi) - zi @ zi) <= 1e-9 * (zi @ zi)
    xx = exact.sample_dense(Q, x)
    np.testing.assert_allclose((Q @ xx.T).T, z, atol=1e-8)
    # the square root is the principal one: x . z > 0 (positive definite map)
    assert np.all(np.einsum("ij,ij->i", x, z) > 0)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", stencil.BCS)
@pytest.mark.parametrize("op", stencil.OPS)
def test_spectral_sample_matches_dense(shape, bc, op):
    Q = stencil.precision_matrix(shape, bc, op, 0.2, tau=0.7, kappa2_prior=KP)
    z = inputs.gaussian_vectors(1, int(np.prod(shape)), seed=11, dtype=np.float64)[0]
    xd = exact.sample_dense(Q, z)[0]
    xs = exact.sample_spectral(shape, bc, op, 0.2, 0.7, z, kappa2_prior=KP)
    np.testing.assert_allclose(xs, xd, rtol=1e-10, atol=1e-10 * np.linalg.norm(xd))


def test_tau_scaling():
    shape = (6, 6)
    Q = stencil.precision_matrix(shape, "neumann", "spde_squared", 0.4, tau=1.0)
    z = inputs.gaussian_vectors(1, 36, seed=1, dtype=np.float64)
    x1 = exact.sample_dense(Q, z)
    x4 = exact.sample_dense(4.0 * Q, z)
    np.testing.assert_allclose(x4, 0.5 * x1, rtol=1e-12)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", stencil.BCS)
@pytest.mark.parametrize("op", stencil.OPS)
def test_logdet_three_routes(shape, bc, op):
    Q = stencil.precision_matrix(shape, bc, op, 0.25, tau=1.9, kappa2_prior=KP)
    ld_chol = exact.logdet_cholesky(Q)
    ld_spec = exact.logdet_spectral(shape, bc, op, 0.25, 1.9, kappa2_prior=KP)
    lu = spla.splu(Q.tocsc())
    ld_lu = float(np.sum(np.log(np.abs(lu.U.diagonal()))))
    assert abs(ld_chol - ld_spec) <= 1e-10 * abs(ld_spec) + 1e-10
    assert abs(ld_lu - ld_spec) <= 1e-9 * abs(ld_spec) + 1e-9


@pytest.mark.parametrize("bc", stencil.BCS)
def test_quadform_log_routes_and_trace(bc):
    shape = (5, 6)
    n = 30
    Q = stencil.precision_matrix(shape, bc, "spde_squared", 0.3, tau=1.0)
    V = inputs.rademacher_vectors(3, n, seed=2, dtype=np.float64)
    qd = exact.quadform_log_dense(Q, V)
    qs = exact.quadform_log_spectral(shape, bc, "spde_squared", 0.3, 1.0, V)
    np.testing.assert_allclose(qd, qs, rtol=1e-10, atol=1e-10)
    # unit-vector probes give the trace exactly: sum_i e_i^T log(Q) e_i = log det Q
    tr = exact.quadform_log_dense(Q, np.eye(n)).sum()
    assert abs(tr - exact.logdet_cholesky(Q)) <= 1e-9 * abs(tr)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", stencil.BCS)
@pytest.mark.parametrize("op", stencil.OPS)
def test_solve_routes(shape, bc, op):
    # x = Q^{-1} b (Section 5.1's mean solve): the sparse LU solution has a
    # vanishing residual under the sparse matvec, and for constant kappa^2 it
    # equals the closed-form spectral solve; a variable kappa^2 field is
    # checked through the residual and x^T Q x = x^T b.
    rng = np.random.default_rng(7)
    n = int(np.prod(shape))
    B = inputs.gaussian_vectors(2, n, seed=13, dtype=np.float64)
    Qc = stencil.precision_matrix(shape, bc, op, 0.3, tau=1.7, kappa2_prior=KP)
    xs = exact.solve_sparse(Qc, B)
    for x, b in zip(xs, B):
        assert np.linalg.norm(Qc @ x - b) <= 1e-11 * np.linalg.norm(b)
        xf = exact.solve_spectral(shape, bc, op, 0.3, 1.7, b, kappa2_prior=KP)
        np.testing.assert_allclose(xf, x, rtol=0, atol=1e-10 * np.linalg.norm(x))
    k2 = rng.uniform(0.05, 1.0, size=shape)
    Qv = stencil.precision_matrix(shape, bc, op, k2, tau=0.6, kappa2_prior=KP)
    xv = exact.solve_sparse(Qv, B[:1])[0]
    assert np.linalg.norm(Qv @ xv - B[0]) <= 1e-11 * np.linalg.norm(B[0])
    assert abs(xv @ (Qv @ xv) - xv @ B[0]) <= 1e-10 * abs(xv @ B[0])


def test_stieltjes_route_matches_dense():
    # the quadrature route against dense eigh on a small variable-kappa^2 grid,
    # with loose spectral bounds (Gershgorin above, min kappa^2 below)
    rng = np.random.default_rng(8)
    shape = (9, 11)
    k2 = rng.uniform(0.05, 1.0, size=shape)
    Q = stencil.precision_matrix(shape, "neumann", "spde_squared", k2, tau=1.3)
    z = inputs.gaussian_vectors(1, 99, seed=3, dtype=np.float64)[0]
    lo = 1.3 * k2.min() ** 2
    hi = 1.3 * (k2.max() + 8.0) ** 2
    x = exact.sample_stieltjes(Q, z, lo, hi)
    xe = exact.sample_dense(Q, z)[0]
    assert np.linalg.norm(x - xe) <= 1e-10 * np.linalg.norm(xe)
