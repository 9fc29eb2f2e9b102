"""Pins for oracle/lanczos.py and oracle/precond.py: Algorithm 1 against the
exact map, exact termination, Theorem 1, Proposition 1, Section 6."""
import numpy as np
import pytest

from oracle import exact, lanczos, precond, stencil
from paper_1312_1476_gb300 import inputs


def _problem(shape=(6, 7), bc="neumann", op="spde_squared", seed=4, tau=1.0):
    rng = np.random.default_rng(seed)
    k2 = rng.uniform(0.05, 0.6, size=shape)
    Q = stencil.precision_matrix(shape, bc, op, k2, tau, kappa2_prior=0.45)
    return k2, Q


@pytest.mark.parametrize("bc", stencil.BCS)
@pytest.mark.parametrize("op", stencil.OPS)
def test_full_krylov_space_reproduces_exact_sample(bc, op):
    shape = (5, 6)
    k2, Q = _problem(shape, bc, op)
    z = inputs.gaussian_vectors(1, 30, seed=9, dtype=np.float64)[0]
    x = lanczos.krylov_sample(lambda v: Q @ v, z, m=30, reorth=True)
    xe = exact.sample_dense(Q, z)[0]
    assert np.linalg.norm(x - xe) <= 1e-10 * np.linalg.norm(xe)


def test_exact_termination_on_k_modes():
    # z = sum of k eigenvectors with distinct eigenvalues: the Krylov space is
    # k-dimensional, so Algorithm 1 breaks down at m = k with the exact x.
    N = 8
    shape = (N, N)
    lam1, U1 = stencil.laplacian_eigen_1d(N, "periodic")
    Q = stencil.precision_matrix(shape, "periodic", "shifted_laplacian", 0.1)
    modes = [(0, 0), (1, 0), (2, 3), (4, 4)]
    z = sum((c + 1.0) * np.kron(U1[:, a], U1[:, b]) for c, (a, b) in enumerate(modes))
    run = lanczos.lanczos(lambda v: Q @ v, z, m=40)
    assert run["breakdown"] and run["m"] == len(modes)
    x = lanczos.sample_from_lanczos(run)
    xe = exact.sample_dense(Q, z)[0]
    assert np.linalg.norm(x - xe) <= 1e-12 * np.linalg.norm(xe)


def test_theorem1_bounds_hold():
    k2, Q = _problem((8, 8), "neumann", "shifted_laplacian")
    ev = np.linalg.eigvalsh(Q.toarray())
    lmin, lmax = ev[0], ev[-1]
    z = inputs.gaussian_vectors(1, 64, seed=1, dtype=np.float64)[0]
    xe = exact.sample_dense(Q, z)[0]
    run = lanczos.lanczos(lambda v: Q @ v, z, m=40, reorth=True)
    for m in range(1, run["m"]):
        xm = lanczos.sample_from_lanczos(run, m)
        err = np.linalg.norm(xe - xm)
        rn = lanczos.cg_residual_norm(run["alpha"][:m], run["beta"][:m], run["znorm"])
        rd = lanczos.cg_residual_direct(lambda v: Q @ v, z, run, m)
        assert abs(rn - rd) <= 1e-8 * np.linalg.norm(z) + 1e-8 * rd
        assert err <= lanczos.posterior_bound(lmin, rn) * (1 + 1e-9) + 1e-12
        assert err <= lanczos.apriori_bound(lmin, lmax, m, np.linalg.norm(z)) * (1 + 1e-9)
        th = lanczos.tm_eigh(run["alpha"][:m], run["beta"][:m])[0]
        assert th[0] >= lmin * (1 - 1e-10) and th[-1] <= lmax * (1 + 1e-10)


@pytest.mark.parametrize("tol", [1e-4, 1e-7, 1e-10])
def test_stopping_rule_meets_tolerance(tol):
    k2, Q = _problem((10, 10), "periodic", "shifted_laplacian", tau=2.0)
    z = inputs.gaussian_vectors(1, 100, seed=2, dtype=np.float64)[0]
    x, m, est, status = lanczos.adaptive_sample(lambda v: Q @ v, z, tol, m_max=100)
    xe = exact.sample_dense(Q, z)[0]
    assert status in ("ok", "breakdown")
    assert np.linalg.norm(x - xe) <= tol * np.linalg.norm(xe)
    assert est <= tol


def test_perfect_preconditioner_collapses():
    # Section 5: with M = Q the preconditioned operator is the identity, u = z
    # and Proposition 1 returns x = M^{-1/2} z after a single step.
    shape = (8, 8)
    for bc, op in (("periodic", "spde_squared"), ("neumann", "spde_squared"),
                   ("dirichlet", "shifted_laplacian")):
        Q = stencil.precision_matrix(shape, bc, op, 0.3, 1.5)
        z = inputs.gaussian_vectors(1, 64, seed=3, dtype=np.float64)[0]
        A = lanczos.preconditioned_operator(Q, shape, bc, op, 0.3, 1.5)
        run = lanczos.lanczos(A, z, m=10)
        assert run["m"] == 1 and run["breakdown"]
        x, m, est, status = lanczos.precond_sample(Q, shape, bc, op, 0.3, 1.5, z, 1e-12, 10)
        xe = exact.sample_dense(Q, z)[0]
        assert m == 1
        assert np.linalg.norm(x - xe) <= 1e-12 * np.linalg.norm(xe)


@pytest.mark.parametrize("kind", ["periodic", "neumann"])
def test_prop1_map_and_covariance(kind):
    shape = (6, 6)
    k2, Q = _problem(shape, "neumann", "spde_squared")
    kb = precond.kappa2_bar(k2)
    A, P = precond.preconditioned_operator_dense(Q, shape, kind, "spde_squared", kb, 1.0)
    # covariance of x = P A^{-1/2} z is P A^{-1} P, which must equal Q^{-1}
    Qinv = np.linalg.inv(Q.toarray())
    np.testing.assert_allclose(P @ np.linalg.inv(A) @ P, Qinv, atol=1e-9 * np.abs(Qinv).max())
    z = inputs.gaussian_vectors(1, 36, seed=8, dtype=np.float64)[0]
    xd = precond.sample_prop1_dense(Q, shape, kind, "spde_squared", kb, 1.0, z)[0]
    assert abs(xd @ (Q @ xd) - z @ z) <= 1e-9 * (z @ z)
    x, m, est, status = lanczos.precond_sample(Q, shape, kind, "spde_squared", kb, 1.0, z,
                                               1e-11, 36, reorth=True)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_prop1_covariance_statistical():
    # many draws through the Krylov map: sample covariance ~ Q^{-1} (5 s.e.)
    shape = (3, 3)
    k2, Q = _problem(shape, "periodic", "shifted_laplacian")
    Z = inputs.gaussian_vectors(4000, 9, seed=21, dtype=np.float64)
    X = np.array([lanczos.krylov_sample(lambda v: Q @ v, z, 9, reorth=True) for z in Z])
    C = X.T @ X / len(X)
    Ce = np.linalg.inv(Q.toarray())
    se = np.sqrt((np.outer(np.diag(Ce), np.diag(Ce)) + Ce ** 2) / len(X))
    assert np.all(np.abs(C - Ce) <= 5 * se)


def test_preconditioned_logdet_sign():
    # Section 6.2 prints log det Q = log det(F^-1 Q F^-T) - 2 log det F; the
    # determinant identity gives + 2 log det F = + log det M.
    shape = (5, 5)
    k2, Q = _problem(shape, "neumann", "spde_squared")
    kb = precond.kappa2_bar(k2)
    A, P = precond.preconditioned_operator_dense(Q, shape, "periodic", "spde_squared", kb, 1.0)
    ldq = exact.logdet_cholesky(Q)
    lda = exact.logdet_cholesky(A)
    ldm = precond.logdet(shape, "periodic", "spde_squared", kb, 1.0)
    assert abs(ldq - (lda + ldm)) <= 1e-9 * abs(ldq)
    assert abs(ldq - (lda - ldm)) > 1.0


def test_quadrature_full_space_is_exact():
    k2, Q = _problem((5, 5), "dirichlet", "shifted_laplacian")
    V = inputs.rademacher_vectors(4, 25, seed=5, dtype=np.float64)
    exact_q = exact.quadform_log_dense(Q, V)
    for v, qe in zip(V, exact_q):
        run = lanczos.lanczos(lambda u: Q @ u, v, m=25, reorth=True)
        q = run["znorm"] ** 2 * lanczos.tm_log_e1e1(run["alpha"], run["beta"])
        assert abs(q - qe) <= 1e-10 * abs(qe)
    # unit-vector probes give log det exactly
    est, se, qs = lanczos.hutchinson_logdet(lambda u: Q @ u, np.eye(25), 1e-13, 25, reorth=True)
    assert abs(25 * est - exact.logdet_cholesky(Q)) <= 1e-9 * abs(exact.logdet_cholesky(Q))


def test_hutchinson_unbiased_statistical():
    k2, Q = _problem((4, 4), "periodic", "spde_squared")
    ld = exact.logdet_cholesky(Q)
    V = inputs.rademacher_vectors(3000, 16, seed=17, dtype=np.float64)
    q = exact.quadform_log_dense(Q, V)
    se = q.std(ddof=1) / np.sqrt(len(q))
    assert abs(q.mean() - ld) <= 4 * se
    # Rademacher variance = 2 sum_{i != j} B_ij^2 with B = log Q
    lam, U = exact.dense_eigh(Q)
    B = (U * np.log(lam)) @ U.T
    var = 2 * (np.sum(B ** 2) - np.sum(np.diag(B) ** 2))
    assert abs(q.var(ddof=1) - var) <= 0.15 * var


@pytest.mark.parametrize("p", [1, 2, 3])
def test_coloured_masks_partition_and_distance(p):
    shape = (12, 12)
    masks = lanczos.coloured_probe_masks(shape, p)
    assert np.all(masks.sum(axis=0) == 1)
    for mk in masks:
        idx = np.nonzero(mk)[0]
        ys, xs = idx // 12, idx % 12
        d = np.abs(ys[:, None] - ys[None, :]) + np.abs(xs[:, None] - xs[None, :])
        np.fill_diagonal(d, 10 ** 6)
        assert d.min() > p


@pytest.mark.parametrize("p", [1, 2])
def test_coloured_estimator_exact_mean_and_variance(p):
    # all 2^9 sign patterns on a 3 x 3 grid: the coloured estimator
    # sum_c v_c^T log(Q) v_c has mean log det Q exactly and variance
    # 2 sum_c sum_{i != j in c} B_ij^2, B = log Q (Section 6.1 with the
    # factor 2 of Rademacher quadratic forms)
    shape = (3, 3)
    Q = stencil.precision_matrix(shape, "neumann", "spde_squared", 0.7, 1.3).toarray()
    ld = exact.logdet_cholesky(Q)
    masks = lanczos.coloured_probe_masks(shape, p)
    signs = np.array([[1.0 if (k >> b) & 1 else -1.0 for b in range(9)] for k in range(2 ** 9)])
    vals = np.zeros(len(signs))
    for mk in masks:
        vals += exact.quadform_log_dense(Q, np.where(mk[None, :], signs, 0.0))
    assert abs(vals.mean() - ld) <= 1e-10 * abs(ld)
    lam, U = exact.dense_eigh(Q)
    B = (U * np.log(lam)) @ U.T
    var = 0.0
    for mk in masks:
        Bc = B[np.ix_(mk, mk)]
        var += 2 * (np.sum(Bc ** 2) - np.sum(np.diag(Bc) ** 2))
    assert abs(vals.var() - var) <= 1e-10 * max(var, 1e-300) + 1e-14


def test_coloured_lanczos_quadrature_matches_dense():
    # the Lanczos-quadrature coloured estimator against dense quadratic forms
    shape = (8, 8)
    Q = stencil.precision_matrix(shape, "periodic", "shifted_laplacian", 0.3, 1.0)
    draws = inputs.rademacher_vectors(3, 64, seed=21, dtype=np.float64)
    est, se, q = lanczos.coloured_hutchinson_logdet(lambda v: Q @ v, shape, 1, draws, 1e-12, 64, reorth=True)
    masks = lanczos.coloured_probe_masks(shape, 1)
    for d in range(3):
        for c, mk in enumerate(masks):
            ref = exact.quadform_log_dense(Q.toarray(), np.where(mk, draws[d], 0.0)[None, :])[0]
            assert abs(q[d, c] - ref) <= 1e-9 * abs(ref) + 1e-9
    assert abs(est - q.sum(axis=1).mean()) <= 1e-12 * abs(est)


def test_cg_exact_termination_and_lanczos_iterates():
    # CG on an operator with k distinct eigenvalues ends in k steps with the
    # exact solution; every CG iterate equals the Lanczos one
    # ||b|| V_k T_k^{-1} e_1 built by the independent Lanczos code.
    rng = np.random.default_rng(2)
    d = np.repeat([0.5, 1.5, 4.0, 9.0], 10)
    rng.shuffle(d)
    b = rng.standard_normal(d.size)
    x, k, st = lanczos.cg_solve(lambda v: d * v, b, tol=1e-13, m_max=40)
    assert st == "ok" and k == 4
    np.testing.assert_allclose(x, b / d, rtol=1e-11)
    k2, Q = _problem((6, 7), "dirichlet", "spde_squared")
    b = inputs.gaussian_vectors(1, 42, seed=3, dtype=np.float64)[0]
    run = lanczos.lanczos(lambda v: Q @ v, b, m=12, reorth=True)
    for m in (3, 7, 12):
        T = lanczos.tridiagonal(run["alpha"][:m], run["beta"][:m])
        y = run["znorm"] * (run["V"][:m].T @ np.linalg.solve(T, np.eye(m)[0]))
        xc, kc, _ = lanczos.cg_solve(lambda v: Q @ v, b, tol=0.0, m_max=m)
        assert kc == m
        np.testing.assert_allclose(xc, y, rtol=0, atol=1e-9 * np.linalg.norm(y))


def test_cg_reaches_the_sparse_solve_with_the_stopping_rule():
    # the relative-residual rule is met, and the error obeys ||e|| / ||x|| <= kappa(Q) tol
    k2, Q = _problem((8, 9), "neumann", "shifted_laplacian")
    b = inputs.gaussian_vectors(1, 72, seed=6, dtype=np.float64)[0]
    xe = exact.solve_sparse(Q, b)[0]
    lam = np.linalg.eigvalsh(Q.toarray())
    for tol in (1e-4, 1e-8, 1e-12):
        x, k, st = lanczos.cg_solve(lambda v: Q @ v, b, tol=tol, m_max=400)
        assert st == "ok"
        assert np.linalg.norm(b - Q @ x) <= tol * np.linalg.norm(b) * (1 + 1e-6)
        assert np.linalg.norm(x - xe) <= (lam[-1] / lam[0]) * tol * np.linalg.norm(xe) * 1.01


def test_lanczos_reference_against_the_stieltjes_route_at_mid_size():
    # The large-grid reference of the GPU parity tests (Algorithm 1 in FP64 with
    # full reorthogonalisation, run to 1e-12) against an independent route, the
    # Stieltjes-integral quadrature with sparse LU solves, on a 64 x 96
    # variable-kappa^2 grid (no closed form, too large for a dense check)
    shape = (64, 96)
    n = 64 * 96
    k2 = inputs.kappa2_uniform_field(shape, seed=1, lo=0.3, hi=1.0)  # kappa(Q) ~ 770: a few hundred steps
    Q = stencil.precision_matrix(shape, "neumann", "spde_squared", k2.astype(np.float64), 1.0)
    z = inputs.gaussian_vectors(1, n, seed=2, dtype=np.float64)[0]
    x_l, m, est, st = lanczos.adaptive_sample(lambda v: Q @ v, z, 1e-12, 3000, reorth=True)
    assert st == "ok"
    x_q = exact.sample_stieltjes(Q, z, float(k2.min()) ** 2, (float(k2.max()) + 8.0) ** 2)
    assert np.linalg.norm(x_l - x_q) <= 1e-9 * np.linalg.norm(x_q)
