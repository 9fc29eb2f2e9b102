"""GPU parity of the sparse (CSR) path with an incomplete-Cholesky
preconditioner (Section 5.2, Figure 3; Proposition 1 with M = F F^T) against
the oracle's dense maps.

The factor F fed to both sides is the oracle's (oracle/sparse.py); the
library's own factorisation is compared with it on the host
(tests/test_sparse_host.py).  Tolerances:
* FP64 at tol 1e-11: relative error of x <= 1e-10 (the stopping rule bounds
  the error of A^{-1/2} z; F^{-T} adds rounding only);
* FP32 at tol 1e-6: relative error <= max(2e-6 + 8 u sqrt(kappa(S)), 64 u kappa(F)),
  u = 2^-24, S the iterated operator (Q, or A = F^{-1} Q F^{-T}): the final
  F^{-T} solve and the applies of F^{-1}, F^{-T} in the step run in FP32,
  whose rounding the condition number of F amplifies; and the FP32 CSR
  product rounds relative to |Q| |x| (a general matrix has no difference form
  like the lattice stencils), a perturbation of S that moves S^{-1/2} z by up
  to about sqrt(kappa(S)) u in the cases here.
  In FP32 the library may instead return NOT_CONVERGED when its accuracy
  check finds the iteration's floor above tol; its error estimate must then
  cover the error, less the rounding of the final F^{-T} map (64 u kappa(F)),
  which comes after the iteration.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from honesty import assert_honest
from oracle import exact, lanczos as olz, sparse as osp
from paper_1312_1476_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def g():
    from paper_1312_1476_gb300 import gmrf
    assert torch.cuda.is_available()
    return gmrf


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / np.linalg.norm(b))


def _q(kind):
    if kind == "figure3":
        return osp.csr(*inputs.figure3_matrix())
    nx, ny, sq = {"lattice": (14, 11, False), "squared": (13, 12, True), "small": (7, 5, True)}[kind]
    return osp.csr(*inputs.random_sparse_spd(nx, ny, seed=21, squared=sq))


def _factor(Q, droptol, shift):
    if droptol == "none":
        return None
    return osp.ichol(Q, droptol=droptol, shift=shift)


def _sample(prob, Z, tol, m_max, precision):
    nvec, n = Z.shape
    x = torch.empty(nvec * n, dtype=torch.float64 if precision == "fp64" else torch.float32, device="cuda")
    rc, info = prob.sample(x, nsamples=nvec, tol=tol, m_max=m_max, z=_dev(Z), check_every=4)
    return rc, info, x.cpu().numpy().reshape(nvec, n)


def _expected(Q, F, Z, tau=1.0):
    Z = Z.astype(np.float64)
    X = exact.sample_dense(Q, Z) if F is None else osp.sample_precond_dense(Q, F, Z)
    return X / np.sqrt(tau)


def _fp32_tol(F, Q):
    S = Q.toarray() if F is None else osp.preconditioned_matrix(Q, F)
    lam = np.linalg.eigvalsh(S)
    lim = 2e-6 + 8 * U32 * np.sqrt(lam[-1] / lam[0])
    if F is not None:
        s = np.linalg.svd(F.toarray(), compute_uv=False)
        lim = max(lim, 64 * U32 * s[0] / s[-1])
    return lim


def _fp32_map_tol(F):
    # rounding of the final FP32 map x = F^{-T} u, which lies outside the
    # iteration's own error estimate
    if F is None:
        return 0.0
    s = np.linalg.svd(F.toarray(), compute_uv=False)
    return 64 * U32 * s[0] / s[-1]


FACTORS = [("none", 0.0), (None, 0.05), (1e-2, 0.1), (1e-4, 0.0), (np.inf, 0.0), (0.0, 0.0)]


@pytest.mark.parametrize("kind", ["lattice", "squared"])
@pytest.mark.parametrize("droptol,shift", FACTORS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sample_vs_prop1_dense(g, kind, droptol, shift, precision):
    Q = _q(kind)
    F = _factor(Q, droptol, shift)
    n = Q.shape[0]
    dt = np.float64 if precision == "fp64" else np.float32
    Z = inputs.gaussian_vectors(3, n, seed=5, dtype=dt)
    tol = 1e-11 if precision == "fp64" else 1e-6
    with g.SparseProblem(Q, F, tau=1.7, precision=precision) as p:
        rc, info, X = _sample(p, Z, tol, 4 * n, precision)
    Xe = _expected(Q, F, Z, tau=1.7)
    lim = 1e-10 if precision == "fp64" else _fp32_tol(F, Q)
    for s in range(3):
        if precision == "fp64":
            assert info[s].status == g.OK
        assert_honest(info[s], _rel(X[s], Xe[s]), lim, slack=_fp32_map_tol(F) if precision == "fp32" else 0.0)


@pytest.mark.parametrize("droptol,shift", [(0.0, 0.0), (1e-5, 1e-4), (1e-3, 1e-3), (None, 0.01)])
def test_figure3_fp64(g, droptol, shift):
    # the Figure 3 matrix (31^2 G)^2 with several factors: parity of x and of
    # the subspace size with the oracle's Algorithm 1 on the same A
    Q = _q("figure3")
    F = osp.ichol(Q, droptol=droptol, shift=shift)
    n = Q.shape[0]
    Z = inputs.gaussian_vectors(2, n, seed=6, dtype=np.float64)
    with g.SparseProblem(Q, F, precision="fp64") as p:
        rc, info, X = _sample(p, Z, 1e-10, 600, "fp64")
    Xe = _expected(Q, F, Z)
    A = osp.preconditioned_matrix(Q, F)
    for s in range(2):
        assert info[s].status == g.OK
        assert _rel(X[s], Xe[s]) <= 1e-9
        _, m_or, _, _ = olz.adaptive_sample(lambda v: A @ v, Z[s], 1e-10, 600, check_every=4)
        assert abs(info[s].m_used - m_or) <= max(4, 0.05 * m_or)


def test_figure3_fp32_good_factor(g):
    Q = _q("figure3")
    F = osp.ichol(Q, droptol=1e-5, shift=1e-4)
    Z = inputs.gaussian_vectors(2, Q.shape[0], seed=6, dtype=np.float32)
    with g.SparseProblem(Q, F, precision="fp32") as p:
        rc, info, X = _sample(p, Z, 1e-6, 200, "fp32")
    Xe = _expected(Q, F, Z)
    for s in range(2):
        assert_honest(info[s], _rel(X[s], Xe[s]), _fp32_tol(F, Q), slack=_fp32_map_tol(F))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_exact_factor_one_step(g, precision):
    # F the exact Cholesky factor: A = I, so one Lanczos step is exact and x = F^{-T} z.
    # In FP64 beta_0 = ||A v_0 - v_0|| is rounding noise far below the breakdown
    # threshold (m = 1).  In FP32 the applies of F^{-T}, Q, F^{-1} leave
    # A v - v at up to kappa(Q) u relative, above the FP32 threshold (1e-6), so
    # a few more steps on the rounding-perturbed identity may run.
    Q = _q("squared")
    F = osp.ichol(Q, droptol=0.0)
    dt = np.float64 if precision == "fp64" else np.float32
    Z = inputs.gaussian_vectors(2, Q.shape[0], seed=8, dtype=dt)
    with g.SparseProblem(Q, F, precision=precision) as p:
        rc, info, X = _sample(p, Z, 1e-8 if precision == "fp64" else 1e-6, 50, precision)
    Xe = osp.apply_upper_inv(F, Z.astype(np.float64))
    for s in range(2):
        assert info[s].status == g.OK and info[s].m_used <= (1 if precision == "fp64" else 4)
        assert _rel(X[s], Xe[s]) <= (1e-12 if precision == "fp64" else _fp32_tol(F, Q))


@pytest.mark.parametrize("droptol,shift", [("none", 0.0), (1e-2, 0.1), (None, 0.05)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_logdet_fixed_probes(g, droptol, shift, precision):
    # per-probe quadratures against q_i = v_i^T log(A) v_i, and the estimate
    # mean(q) + 2 sum log F_ii + n log tau
    Q = _q("lattice")
    F = _factor(Q, droptol, shift)
    n = Q.shape[0]
    dt = np.float64 if precision == "fp64" else np.float32
    V = inputs.rademacher_vectors(6, n, seed=9, dtype=dt)
    tau = 2.5
    with g.SparseProblem(Q, F, tau=tau, precision=precision) as p:
        ld, se, q, info, rc = p.logdet(nprobes=6, tol=1e-10 if precision == "fp64" else 1e-6, m_max=4 * n,
                                       probes=_dev(V), check_every=4)
    if F is None:
        qe = exact.quadform_log_dense(Q, V.astype(np.float64))
        shift_e = 0.0
    else:
        qe = osp.quadform_log_precond(Q, F, V.astype(np.float64))
        shift_e = osp.logdet_factor(F)
    rt = 1e-8 if precision == "fp64" else 2e-4
    np.testing.assert_allclose(q, qe, rtol=rt, atol=rt * np.abs(qe).max())
    np.testing.assert_allclose(ld, qe.mean() + shift_e + n * np.log(tau), rtol=rt)
    np.testing.assert_allclose(se, qe.std(ddof=1) / np.sqrt(6), rtol=1e-3 if precision == "fp64" else 5e-2)


def test_logdet_unit_probes_give_exact_logdet(g):
    # all n unit vectors as probes: the estimate is tr log A + log det(F F^T) = log det Q
    Q = _q("small")
    F = osp.ichol(Q, droptol=1e-2, shift=0.1)
    n = Q.shape[0]
    V = np.eye(n)
    with g.SparseProblem(Q, F, precision="fp64") as p:
        ld, se, q, info, rc = p.logdet(nprobes=n, tol=1e-12, m_max=4 * n, probes=_dev(V), check_every=2)
    # the library returns mean(q) + log det(F F^T), and n mean(q) = tr log A
    np.testing.assert_allclose((ld - osp.logdet_factor(F)) * n + osp.logdet_factor(F),
                               exact.logdet_cholesky(Q), rtol=1e-9)


@pytest.mark.parametrize("droptol,shift", [("none", 0.0), (1e-2, 0.1)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_solve_vs_sparse_lu(g, droptol, shift, precision):
    Q = _q("squared")
    F = _factor(Q, droptol, shift)
    n = Q.shape[0]
    tau = 0.7
    dt = np.float64 if precision == "fp64" else np.float32
    B = inputs.gaussian_vectors(2, n, seed=10, dtype=dt)
    tol = 1e-11 if precision == "fp64" else 1e-6
    x = torch.empty(2 * n, dtype=torch.float64 if precision == "fp64" else torch.float32, device="cuda")
    with g.SparseProblem(Q, F, tau=tau, precision=precision) as p:
        rc, info = p.solve(_dev(B), x, nrhs=2, tol=tol, m_max=6 * n, check_every=4)
    X = x.cpu().numpy().reshape(2, n)
    Xe = exact.solve_sparse(tau * Q, B.astype(np.float64))
    S = Q.toarray() if F is None else osp.preconditioned_matrix(Q, F)
    lam = np.linalg.eigvalsh(S)
    kap = lam[-1] / lam[0]
    for s in range(2):
        assert info[s].status == g.OK
        lim = kap * tol * 2 if precision == "fp64" else max(kap * tol * 2, 64 * U32 * kap)
        if F is not None and precision == "fp32":
            lim = max(lim, _fp32_tol(F, Q) * np.sqrt(kap))
        assert _rel(X[s], Xe[s]) <= lim


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_apply_modes(g, precision):
    Q = _q("squared")
    F = osp.ichol(Q, droptol=1e-2, shift=0.1)
    n = Q.shape[0]
    tau = 1.3
    dt = np.float64 if precision == "fp64" else np.float32
    V = inputs.gaussian_vectors(3, n, seed=12, dtype=dt)
    Vd = V.astype(np.float64)
    A = osp.preconditioned_matrix(Q, F)
    want = {0: tau * (Q @ Vd.T).T, 1: (A @ Vd.T).T, 2: osp.apply_upper_inv(F, Vd) / np.sqrt(tau)}
    rt = 1e-12 if precision == "fp64" else 20 * _fp32_tol(F, Q)
    with g.SparseProblem(Q, F, tau=tau, precision=precision) as p:
        for which in (0, 1, 2):
            y = torch.empty(3 * n, dtype=torch.float64 if precision == "fp64" else torch.float32, device="cuda")
            p.apply(which, _dev(V), y, nvec=3)
            Y = y.cpu().numpy().reshape(3, n)
            for s in range(3):
                assert _rel(Y[s], want[which][s]) <= rt


def test_batch_equals_alone(g):
    Q = _q("squared")
    F = osp.ichol(Q, droptol=1e-2, shift=0.1)
    n = Q.shape[0]
    Z = inputs.gaussian_vectors(9, n, seed=14, dtype=np.float32)
    with g.SparseProblem(Q, F, precision="fp32") as p:
        _, info_all, X_all = _sample(p, Z, 1e-6, 4 * n, "fp32")
        _, info_one, X_one = _sample(p, Z[4:5], 1e-6, 4 * n, "fp32")
    np.testing.assert_array_equal(X_all[4], X_one[0])
    assert info_all[4].m_used == info_one[0].m_used


def test_device_noise_and_tau_scaling(g):
    # the library's own Philox z, and x(tau Q) = tau^{-1/2} x(Q) bitwise up to one rounding
    Q = _q("lattice")
    F = osp.ichol(Q, droptol=1e-2)
    n = Q.shape[0]
    xs = []
    for tau in (1.0, 4.0):
        x = torch.empty(2 * n, dtype=torch.float64, device="cuda")
        with g.SparseProblem(Q, F, tau=tau, precision="fp64") as p:
            rc, info = p.sample(x, nsamples=2, tol=1e-11, m_max=4 * n, seed=17)
            assert rc == g.OK
        xs.append(x.cpu().numpy().reshape(2, n))
    np.testing.assert_allclose(xs[1], xs[0] / 2.0, rtol=1e-14, atol=1e-15)
    # and parity against the oracle for that z
    from oracle import philox
    Z = philox.gaussian(2, n, 17)
    np.testing.assert_allclose(xs[0], _expected(Q, F, Z), rtol=0, atol=1e-10 * np.abs(xs[0]).max())


def test_one_by_one_and_diagonal(g):
    # n = 1: x = z / sqrt(tau q); a diagonal Q with F = its square root: A = I
    for n, vals in ((1, [4.0]), (5, [1.0, 2.0, 3.0, 4.0, 5.0])):
        rp = np.arange(n + 1, dtype=np.int64)
        ci = np.arange(n, dtype=np.int32)
        va = np.array(vals, dtype=np.float64)
        Fv = np.sqrt(va)
        Z = inputs.gaussian_vectors(2, n, seed=1, dtype=np.float64)
        for F in (None, (rp, ci, Fv)):
            with g.SparseProblem((rp, ci, va), F, tau=2.0, precision="fp64") as p:
                rc, info, X = _sample(p, Z, 1e-12, 10, "fp64")
            np.testing.assert_allclose(X, Z / np.sqrt(2.0 * va), rtol=1e-14)
            # A = I with the factor (or n = 1): one step; Q = diag(1..5) alone: at most n
            for i in info:
                assert i.m_used <= n
                if F is not None or n == 1:
                    assert i.m_used == 1


def test_validation(g):
    Q = _q("small")
    Q.sort_indices()
    rp, ci, va = Q.indptr.astype(np.int64), Q.indices.astype(np.int32), Q.data.copy()
    F = osp.ichol(Q, droptol=1e-2, shift=0.1)
    # asymmetric Q
    va2 = va.copy()
    va2[1] *= 2.0
    with pytest.raises(g.GmrfError) as e:
        g.SparseProblem((rp, ci, va2), None)
    assert e.value.code == g.ERR_INVALID
    # F with an entry above the diagonal
    Fu = (F + sp.csr_matrix(([0.5], ([0], [3])), shape=F.shape)).tocsr()
    with pytest.raises(g.GmrfError) as e:
        g.SparseProblem(Q, Fu)
    assert e.value.code == g.ERR_INVALID
    # F with a missing diagonal entry
    Fd = F.tolil()
    Fd[2, 2] = 0.0
    Fd = Fd.tocsr()
    Fd.eliminate_zeros()
    with pytest.raises(g.GmrfError) as e:
        g.SparseProblem(Q, Fd)
    assert e.value.code == g.ERR_INVALID
    # beyond the shared-memory limit of one block (FP64)
    n = 40000
    big = (np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n))
    with pytest.raises(g.GmrfError) as e:
        g.SparseProblem(big, None, precision="fp64")
    assert e.value.code == g.ERR_UNSUPPORTED
    # unsupported options
    with g.SparseProblem(Q, F, precision="fp32") as p:
        x = torch.empty(Q.shape[0], dtype=torch.float32, device="cuda")
        rc, _ = p.sample(x, raise_on_error=False, v_storage="bf16")
        assert rc == g.ERR_UNSUPPORTED
        rc, _ = p.sample(x, raise_on_error=False, v_storage="none")
        assert rc == g.ERR_UNSUPPORTED
        _, _, _, _, rc = p.logdet(nprobes=2, colour_dist=1, raise_on_error=False)
        assert rc == g.ERR_UNSUPPORTED
        y = torch.empty_like(x)
        assert g.lib().gmrf_apply_inv_sqrt_noalloc(p._h, 1, g._ptr(x), g._ptr(y)) == g.ERR_UNSUPPORTED
    with g.SparseProblem(Q, None, precision="fp32") as p:
        x = torch.ones(Q.shape[0], dtype=torch.float32, device="cuda")
        y = torch.empty_like(x)
        assert g.lib().gmrf_apply(p._h, 1, 1, g._ptr(x), g._ptr(y)) == g.ERR_INVALID


def test_async_and_sample_logdet_equal_synchronous(g):
    Q = _q("lattice")
    F = osp.ichol(Q, droptol=1e-2)
    n = Q.shape[0]
    with g.SparseProblem(Q, F, precision="fp32") as p:
        x1 = torch.empty(3 * n, dtype=torch.float32, device="cuda")
        x2 = torch.empty_like(x1)
        x3 = torch.empty_like(x1)
        p.sample(x1, nsamples=3, seed=4)
        t = p.submit_sample(x2, nsamples=3, seed=4)
        assert t.wait()[0] == g.OK
        ld, se, q, _, _ = p.logdet(nprobes=4, seed=5)
        rc, _, ld2, se2, q2, _ = p.sample_logdet(x3, nsamples=3, nprobes=4, seed=4, probe_seed=5)
    assert torch.equal(x1, x2) and torch.equal(x1, x3)
    np.testing.assert_array_equal(q, q2)
    assert ld == ld2
