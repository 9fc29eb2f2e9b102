"""GPU parity of the linear solve x = Q^{-1} b (Section 5.1: the sMMALA
proposal mean, solved with the sampler's iteration and preconditioner).

The library returns the Lanczos form of the conjugate-gradient iterate,
x_m = ||b~|| V_m T_m^{-1} e_1, stopped when the relative residual of the
iterated system (Q~ x = b, or A u = M^{-1/2} b with a preconditioner) falls
to tol.  The oracle gives the exact solution (sparse LU) and its own
Hestenes-Stiefel CG on the same system.  Bounds used below:
* the iterate's relative error is at most kappa(S) times its relative
  residual, S the iterated operator (kappa from a dense eigensolve);
* in FP64 the true residual of the iterated system equals the estimate the
  recurrence reports (same quantity, rounding ~1e-16 kappa m), and m equals
  the step count of the oracle's Hestenes-Stiefel CG within max(1, 5% of m):
  the two forms agree in exact arithmetic and within one step for the
  well-conditioned systems (kappa <= 10); with outlying eigenvalues (a
  Dirichlet grid under the torus preconditioner, kappa ~ 500) or kappa ~ 1e4
  the delay that lost orthogonality causes depends on the rounding itself
  (the oracle's own count moves by 5 steps at m ~ 1400 between a sparse and
  a dense matvec), a few percent of m;
* in FP32 the recurrence's residual is not the attainable true residual
  (FP32 operator applies), so FP32 parity is the error bound, with an FP32
  floor of 64 u kappa(S), u = 2^-24.
"""
import numpy as np
import pytest

from oracle import exact, lanczos as olz, precond, stencil
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


def _setup(shape, bc, op, pre, lgcp=False):
    """Q (oracle), the iterated operator S (dense), b -> b~, and the problem kwargs."""
    if lgcp:
        mdl = inputs.lgcp_smmala_model(shape[0])
        k2, tau, kb = mdl["d"], mdl["tau"], mdl["kappa2_prior"]
        Q = stencil.precision_matrix(shape, bc, op, k2.astype(np.float64), tau, kappa2_prior=kb)
        kw = dict(kappa2=_dev(k2), kappa2_const=kb, tau=tau)
        pop = "spde_squared"  # the prior's symbol (Theorem 2's preconditioner)
    else:
        k2 = inputs.kappa2_gp_field(shape, seed=1, ell=shape[0] / 8.0)
        tau = 2.0
        Q = stencil.precision_matrix(shape, bc, op, k2.astype(np.float64), tau)
        kb = precond.kappa2_bar(k2)
        kw = dict(kappa2=_dev(k2), tau=tau)
        if pre != "none":
            kw["kappa2_precond"] = kb
        pop = op
    if pre == "none":
        S = Q.toarray() / tau
        bt = lambda b: b
        sres = lambda x, b: np.linalg.norm(b - Q @ x) / np.linalg.norm(b)
    else:
        okind = "periodic" if pre == "circulant" else "neumann"
        S, _ = precond.preconditioned_operator_dense(Q, shape, okind, pop, kb, tau)
        P = lambda v: precond.apply_power(shape, okind, pop, kb, tau, v, -0.5)
        bt = P
        sres = lambda x, b: np.linalg.norm(P(b - Q @ x)) / np.linalg.norm(P(b))
    lam = np.linalg.eigvalsh(S)
    return Q, S, lam[-1] / lam[0], bt, sres, kw


CASES = [((32, 64), bc, op, pre, False)
         for op in ("shifted_laplacian", "spde_squared")
         for bc, pre in (("periodic", "none"), ("neumann", "none"), ("dirichlet", "none"),
                         ("periodic", "circulant"), ("neumann", "mirror"), ("dirichlet", "circulant"))]
CASES += [((32, 32), "periodic", "spde_plus_diag", "circulant", True),
          ((32, 32), "periodic", "spde_plus_diag", "none", True)]


@pytest.mark.parametrize("shape,bc,op,pre,lgcp", CASES)
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_solve_vs_oracle(g, shape, bc, op, pre, lgcp, precision):
    n = int(np.prod(shape))
    Q, S, kap, bt, sres, kw = _setup(shape, bc, op, pre, lgcp)
    dt = np.float64 if precision == "fp64" else np.float32
    B = inputs.gaussian_vectors(2, n, seed=5, dtype=dt)
    tol = 1e-8 if precision == "fp64" else 1e-6
    with g.Problem(shape, bc, op, precond=pre, precision=precision, **kw) as p:
        x = torch.empty(2 * n, dtype=torch.from_numpy(B).dtype, device="cuda")
        rc, info = p.solve(_dev(B), x, nrhs=2, tol=tol, m_max=3000)
        X = x.cpu().numpy().reshape(2, n)
    assert rc == g.OK
    xe = exact.solve_sparse(Q, B.astype(np.float64))
    for s in range(2):
        assert info[s].err_est <= tol
        floor = 0.0 if precision == "fp64" else 64 * U32 * kap
        assert _rel(X[s], xe[s]) <= kap * tol * 1.01 + floor
        if precision == "fp64":
            b = B[s].astype(np.float64)
            r = sres(X[s], b)
            assert abs(r - info[s].err_est) <= 1e-3 * info[s].err_est + 1e-13 * kap
            _, m_or, st = olz.cg_solve(lambda v: S @ v, bt(b), tol, 3000)
            assert st == "ok" and abs(info[s].m_used - m_or) <= max(1, 0.05 * m_or)


def test_solve_batch_invariant_host_pointers_zero_and_limits(g):
    shape = (64, 64)
    n = 4096
    k2 = inputs.kappa2_gp_field(shape, seed=2, ell=8.0)
    B = inputs.gaussian_vectors(5, n, seed=9, dtype=np.float32)
    B[3] = 0.0  # a zero right-hand side: x = 0, m = 0, status OK
    with g.Problem(shape, "neumann", "spde_squared", kappa2=_dev(k2), precond="mirror") as p:
        xb = torch.empty(5 * n, device="cuda")
        rc, info = p.solve(_dev(B), xb, nrhs=5, tol=1e-6, m_max=500)
        assert rc == g.OK
        XB = xb.cpu().numpy().reshape(5, n)
        assert info[3].m_used == 0 and info[3].status == g.OK and not XB[3].any()
        for s in (0, 4):
            # alone and in a batch: the same arithmetic (fixed-order reductions)
            x1 = torch.empty(n, device="cuda")
            rc1, i1 = p.solve(_dev(B[s]), x1, nrhs=1, tol=1e-6, m_max=500)
            assert rc1 == g.OK and i1[0].m_used == info[s].m_used
            assert np.array_equal(x1.cpu().numpy(), XB[s])
        # host buffers in and out
        xh = np.zeros((5, n), dtype=np.float32)
        rc2, _ = p.solve(B, xh, nrhs=5, tol=1e-6, m_max=500)
        assert rc2 == g.OK and np.array_equal(xh, XB)
        # too few steps: NOT_CONVERGED, x_m still written, estimate above tol
        xs = torch.empty(n, device="cuda")
        rc3, i3 = p.solve(_dev(B[0]), xs, nrhs=1, tol=1e-10, m_max=3, raise_on_error=False)
        assert rc3 == g.ERR_NOT_CONVERGED and i3[0].m_used == 3 and i3[0].err_est > 1e-10
        assert np.isfinite(xs.cpu().numpy()).all()
        for bad in (dict(tol=0.0), dict(tol=float("nan")), dict(m_max=0), dict(m_max=9000), dict(nrhs=0)):
            kw = dict(nrhs=1, tol=1e-6, m_max=10)
            kw.update(bad)
            with pytest.raises(g.GmrfError):
                p.solve(_dev(B[0]), xs, **kw)


def test_solve_table1_steps_flat_with_the_prior_preconditioner(g):
    # Section 5.1: one preconditioner (the prior) serves both the proposal's
    # sample and its mean solve; the solve's steps at tol 1e-8 stay flat over
    # the grid while the unpreconditioned count grows
    ms_pre, ms_un = {}, {}
    for N in (16, 32, 64, 128, 256, 512):
        mdl = inputs.lgcp_smmala_model(N)
        b = inputs.gaussian_vectors(1, N * N, seed=4, dtype=np.float64)
        kw = dict(kappa2=_dev(mdl["d"]), kappa2_const=mdl["kappa2_prior"], tau=mdl["tau"], precision="fp64")
        with g.Problem((N, N), "periodic", "spde_plus_diag", precond="circulant", **kw) as p:
            x = torch.empty(N * N, dtype=torch.float64, device="cuda")
            rc, info = p.solve(_dev(b), x, nrhs=1, tol=1e-8, m_max=200)
            assert rc == g.OK
            ms_pre[N] = info[0].m_used
        if N <= 64:
            with g.Problem((N, N), "periodic", "spde_plus_diag", **kw) as p:
                x = torch.empty(N * N, dtype=torch.float64, device="cuda")
                rc, info = p.solve(_dev(b), x, nrhs=1, tol=1e-8, m_max=8000)
                assert rc == g.OK
                ms_un[N] = info[0].m_used
    assert max(ms_pre.values()) - min(ms_pre.values()) <= 1 and max(ms_pre.values()) <= 10
    assert ms_un[16] < ms_un[32] < ms_un[64] and ms_un[64] > 20 * max(ms_pre.values())
