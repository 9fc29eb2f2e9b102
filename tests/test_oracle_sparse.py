"""Pins for oracle/sparse.py: the incomplete Cholesky factor of Section 5.2 and
the preconditioned sampling map of Proposition 1 with M = F F^T."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import exact, lanczos as olz, sparse as osp, stencil
from paper_1312_1476_gb300 import inputs


def _random_q(nx=7, ny=6, squared=False, seed=11):
    return osp.csr(*inputs.random_sparse_spd(nx, ny, seed=seed, squared=squared))


def test_figure3_input_matches_lattice_assembly():
    # the CSR input is the oracle's own Kronecker-sum assembly of (31^2 G)^2
    Q = osp.csr(*inputs.figure3_matrix())
    Qs = stencil.precision_matrix((30, 30), "dirichlet", "spde_squared", 0.0, tau=961.0 ** 2)
    assert abs(Q - Qs).max() == 0.0


@pytest.mark.parametrize("squared", [False, True])
def test_random_input_is_spd_and_symmetric(squared):
    Q = _random_q(squared=squared).toarray()
    np.testing.assert_array_equal(Q, Q.T)
    assert np.linalg.eigvalsh(Q)[0] > 0.0


@pytest.mark.parametrize("squared", [False, True])
def test_zero_droptol_is_exact_cholesky(squared):
    Q = _random_q(squared=squared)
    F = osp.ichol(Q, droptol=0.0).toarray()
    np.testing.assert_allclose(F, np.linalg.cholesky(Q.toarray()), rtol=0, atol=1e-12 * np.abs(F).max())


def test_figure3_zero_droptol_is_exact_cholesky():
    Q = osp.csr(*inputs.figure3_matrix())
    F = osp.ichol(Q, droptol=0.0).toarray()
    L = np.linalg.cholesky(Q.toarray())
    np.testing.assert_allclose(F, L, rtol=0, atol=1e-10 * np.abs(L).max())


def test_ic0_on_tridiagonal_is_exact():
    # no fill-in exists, so IC(0) is the Cholesky factor (a textbook case)
    n = 40
    rng = np.random.default_rng(4)
    off = -rng.uniform(0.1, 1.0, n - 1)
    d = np.zeros(n)
    d[:-1] += -off
    d[1:] += -off
    d += rng.uniform(0.1, 1.0, n)
    T = sp.diags([off, d, off], [-1, 0, 1]).tocsr()
    F = osp.ichol(T, droptol=None).toarray()
    np.testing.assert_allclose(F, np.linalg.cholesky(T.toarray()), rtol=1e-13, atol=1e-14)


def _check_drop_rule(A, F, droptol):
    """F F^T == A on the kept lower pattern; each dropped position's update
    w_i = A_ij - (F F^T)_ij is below droptol ||A[j:, j]||_1 (from F and A alone)."""
    Ad = A.toarray() if sp.issparse(A) else A
    Fd = F.toarray()
    R = Ad - Fd @ Fd.T
    n = Ad.shape[0]
    kept = np.tril(Fd != 0.0)
    scale = np.abs(Ad).max()
    assert np.abs(R[kept]).max() <= 1e-11 * scale
    for j in range(n):
        thr = droptol * np.abs(Ad[j:, j]).sum() if droptol is not None else None
        for i in range(j + 1, n):
            if Fd[i, j] == 0.0:
                if droptol is None:
                    assert Ad[i, j] == 0.0  # IC(0): only positions outside Q's pattern are empty
                else:
                    assert abs(R[i, j]) < thr * (1 + 1e-12) + 1e-12 * scale


@pytest.mark.parametrize("droptol,shift", [(None, 0.0), (1e-2, 0.05), (1e-1, 0.1), (1e-3, 0.1)])
def test_kept_pattern_reproduces_matrix_and_dropped_are_small(droptol, shift):
    Q = _random_q(squared=True)
    F = osp.ichol(Q, droptol=droptol, shift=shift)
    A = Q + shift * sp.diags(Q.diagonal())
    _check_drop_rule(A, F, droptol)


def test_figure3_ict_drop_rule():
    Q = osp.csr(*inputs.figure3_matrix())
    F = osp.ichol(Q, droptol=1e-3, shift=1e-3)
    A = Q + 1e-3 * sp.diags(Q.diagonal())
    _check_drop_rule(A, F, 1e-3)


def test_infinite_droptol_is_jacobi():
    Q = _random_q(squared=True)
    F = osp.ichol(Q, droptol=np.inf)
    np.testing.assert_allclose(F.toarray(), np.diag(np.sqrt(Q.diagonal())), rtol=1e-15)


def test_ic0_figure3_breaks_down_without_shift():
    # (31^2 G)^2 is not an M-matrix; IC(0) meets a negative pivot there
    Q = osp.csr(*inputs.figure3_matrix())
    with pytest.raises(osp.NotFactorable):
        osp.ichol(Q, droptol=None)


@pytest.mark.parametrize("droptol,shift", [(None, 0.0), (1e-2, 0.05), (np.inf, 0.0), (0.0, 0.0)])
def test_sampling_map_has_covariance_q_inverse(droptol, shift):
    # S = F^{-T} A^{-1/2}: S S^T = F^{-T} A^{-1} F^{-1} = (F A F^T)^{-1} = Q^{-1}
    Q = _random_q(squared=True)
    F = osp.ichol(Q, droptol=droptol, shift=shift)
    n = Q.shape[0]
    S = osp.sample_precond_dense(Q, F, np.eye(n)).T  # columns S e_i
    np.testing.assert_allclose(S @ S.T, np.linalg.inv(Q.toarray()), rtol=1e-9, atol=1e-9 * np.abs(S @ S.T).max())


def test_exact_factor_gives_identity_operator():
    Q = _random_q(squared=True)
    F = osp.ichol(Q, droptol=0.0)
    A = osp.preconditioned_matrix(Q, F)
    np.testing.assert_allclose(A, np.eye(A.shape[0]), atol=1e-10)
    z = np.random.default_rng(5).standard_normal(Q.shape[0])
    x = osp.sample_precond_dense(Q, F, z)[0]
    np.testing.assert_allclose(x, osp.apply_upper_inv(F, z)[0], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("droptol,shift", [(None, 0.0), (1e-2, 0.0), (np.inf, 0.0)])
def test_logdet_identity(droptol, shift):
    Q = _random_q(squared=False)
    F = osp.ichol(Q, droptol=droptol, shift=shift)
    np.testing.assert_allclose(osp.logdet_precond(Q, F), exact.logdet_cholesky(Q), rtol=1e-12)


def test_quadform_unit_probes_give_the_trace():
    # sum over e_i of e_i^T log(A) e_i = tr log A = log det A (all n unit vectors)
    Q = _random_q(squared=False)
    F = osp.ichol(Q, droptol=1e-2)
    n = Q.shape[0]
    q = osp.quadform_log_precond(Q, F, np.eye(n))
    np.testing.assert_allclose(q.sum() + osp.logdet_factor(F), exact.logdet_cholesky(Q), rtol=1e-12)


def test_triangular_helpers_invert_the_factor():
    Q = _random_q(squared=True)
    F = osp.ichol(Q, droptol=1e-2, shift=0.05)
    v = np.random.default_rng(8).standard_normal((3, Q.shape[0]))
    np.testing.assert_allclose((F @ osp.apply_lower_inv(F, v).T).T, v, atol=1e-10)
    np.testing.assert_allclose((F.T @ osp.apply_upper_inv(F, v).T).T, v, atol=1e-10)


@pytest.mark.parametrize("droptol,shift", [(None, 0.01), (1e-3, 1e-3)])
def test_krylov_route_matches_dense_map_figure3(droptol, shift):
    # an independent route to the same x: Algorithm 1 (FP64, full reorthogonalisation)
    # on A = F^{-1} Q F^{-T}, then F^{-T}, against the dense eigendecomposition map
    Q = osp.csr(*inputs.figure3_matrix())
    F = osp.ichol(Q, droptol=droptol, shift=shift)
    A = osp.preconditioned_matrix(Q, F)
    z = inputs.gaussian_vectors(1, Q.shape[0], seed=6, dtype=np.float64)[0]
    u, m, _, _ = olz.adaptive_sample(lambda v: A @ v, z, 1e-12, 600, reorth=True)
    x = osp.apply_upper_inv(F, u)[0]
    xe = osp.sample_precond_dense(Q, F, z)[0]
    assert np.linalg.norm(x - xe) <= 1e-10 * np.linalg.norm(xe)
    assert m < 200
