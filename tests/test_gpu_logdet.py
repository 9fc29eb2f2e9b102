"""GPU parity of gmrf_logdet (Section 6 Hutchinson estimator with Lanczos /
Gauss quadrature; Section 6.2 preconditioned split) against the oracle."""
import numpy as np
import pytest

from oracle import exact, lanczos as olz, precond, stencil
from paper_1312_1476_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    from paper_1312_1476_gb300 import gmrf
    assert torch.cuda.is_available()
    return gmrf


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,bc,op", [((12, 10), "neumann", "spde_squared"),
                                         ((14, 14), "periodic", "shifted_laplacian"),
                                         ((5, 6, 7), "dirichlet", "shifted_laplacian")])
def test_fixed_probes_match_exact_quadforms(g, precision, shape, bc, op):
    n = int(np.prod(shape))
    k2 = inputs.kappa2_uniform_field(shape, seed=2, lo=0.1, hi=1.0)
    tau = 1.7
    Q = stencil.precision_matrix(shape, bc, op, k2.astype(np.float64), tau=tau)
    dt = np.float64 if precision == "fp64" else np.float32
    V = inputs.rademacher_vectors(6, n, seed=3, dtype=dt)
    with g.Problem(shape, bc, op, kappa2=_dev(k2), tau=tau, precision=precision) as p:
        ld, se, q, info, rc = p.logdet(nprobes=6, tol=1e-10 if precision == "fp64" else 1e-6, m_max=n,
                                       probes=_dev(V))
    # the library's q_i are for Q / tau (tau enters as n log tau)
    qe = exact.quadform_log_dense(Q / tau, V.astype(np.float64))
    rtol = 1e-8 if precision == "fp64" else 1e-6
    np.testing.assert_allclose(q, qe, rtol=rtol, atol=rtol * np.abs(qe).max())
    est = qe.mean() + n * np.log(tau)
    assert abs(ld - est) <= rtol * abs(est) + rtol
    assert abs(se - qe.std(ddof=1) / np.sqrt(6)) <= 1e-6 * abs(se) + 1e-6


@pytest.mark.parametrize("kind", ["circulant", "mirror"])
def test_preconditioned_logdet_split(g, kind):
    shape = (16, 16)
    n = 256
    k2 = inputs.kappa2_gp_field(shape, seed=1, ell=4.0)
    kb = precond.kappa2_bar(k2)
    tau = 2.0
    okind = "periodic" if kind == "circulant" else "neumann"
    Q = stencil.precision_matrix(shape, "neumann", "spde_squared", k2.astype(np.float64), tau=tau)
    A, P = precond.preconditioned_operator_dense(Q, shape, okind, "spde_squared", kb, tau)
    V = inputs.rademacher_vectors(8, n, seed=5, dtype=np.float64)
    with g.Problem(shape, "neumann", "spde_squared", kappa2=_dev(k2), tau=tau, precond=kind, kappa2_precond=kb,
                   precision="fp64") as p:
        ld, se, q, info, rc = p.logdet(nprobes=8, tol=1e-11, m_max=256, probes=_dev(V))
    qe = exact.quadform_log_dense(A, V)
    np.testing.assert_allclose(q, qe, rtol=1e-8, atol=1e-8 * np.abs(qe).max())
    ldm = precond.logdet(shape, okind, "spde_squared", kb, tau)
    assert abs(ld - (qe.mean() + ldm)) <= 1e-8 * abs(ld)
    # and the split estimates the true log det within its standard error
    assert abs(ld - exact.logdet_cholesky(Q)) <= 5 * se + 1e-6


def test_device_probes_unbiased(g):
    shape = (8, 8)
    k2 = inputs.kappa2_uniform_field(shape, seed=3, lo=0.2, hi=1.0)
    Q = stencil.precision_matrix(shape, "periodic", "spde_squared", k2.astype(np.float64))
    with g.Problem(shape, "periodic", "spde_squared", kappa2=_dev(k2), precision="fp64") as p:
        ld, se, q, info, rc = p.logdet(nprobes=2000, tol=1e-9, m_max=64, seed=11)
    from oracle import philox
    V = philox.rademacher(2000, 64, 11)
    np.testing.assert_allclose(q, exact.quadform_log_dense(Q, V), rtol=1e-7, atol=1e-7)
    assert abs(ld - exact.logdet_cholesky(Q)) <= 4 * se


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("p_dist", [1, 2])
def test_coloured_estimator_matches_oracle(g, precision, p_dist):
    # coloured Hutchinson (Section 6.1) with device probes: each colour-class
    # quadrature against the oracle's estimator on its restated Philox draws
    from oracle import philox
    shape = (24, 24)
    n = 576
    Q = stencil.precision_matrix(shape, "periodic", "shifted_laplacian", 0.3, 1.0)
    ndraw, seed = 3, 4242
    with g.Problem(shape, "periodic", "shifted_laplacian", kappa2_const=0.3, precision=precision) as p:
        tol = 1e-10 if precision == "fp64" else 1e-6
        ld, se, q, info, rc = p.logdet(nprobes=ndraw, tol=tol, m_max=n, seed=seed, colour_dist=p_dist)
    assert rc == g.OK
    ncol = (p_dist + 1) ** 2
    assert len(q) == ndraw * ncol
    draws = philox.rademacher(ndraw, n, seed).astype(np.float64)
    est, se_o, qo = olz.coloured_hutchinson_logdet(lambda v: Q @ v, shape, p_dist, draws, 1e-11, n, reorth=True)
    rtol = 1e-8 if precision == "fp64" else 2e-6
    np.testing.assert_allclose(q.reshape(ndraw, ncol), qo, rtol=rtol, atol=rtol * np.abs(qo).max())
    assert abs(ld - est) <= rtol * abs(est)
    assert abs(se - se_o) <= 1e-6 * se_o + rtol * abs(est)


def test_coloured_estimator_unbiased_and_lower_variance(g):
    # same device draws, plain vs coloured (p = 1, 2): both within 4 standard
    # errors of the exact log det, and the coloured one has the smaller spread
    shape = (32, 32)
    Q = stencil.precision_matrix(shape, "periodic", "shifted_laplacian", 0.2, 1.0)
    ld_exact = exact.logdet_spectral(shape, "periodic", "shifted_laplacian", 0.2, 1.0)
    ses = []
    with g.Problem(shape, "periodic", "shifted_laplacian", kappa2_const=0.2, precision="fp64") as p:
        for pd in (0, 1, 2):
            ld, se, q, info, rc = p.logdet(nprobes=200, tol=1e-9, m_max=400, seed=99, colour_dist=pd)
            assert rc == g.OK
            assert abs(ld - ld_exact) <= 4 * se
            ses.append(se)
    assert ses[1] < 0.7 * ses[0] and ses[2] < ses[1]


@pytest.mark.parametrize("colour_dist", [0, 1])
@pytest.mark.parametrize("block_width", [0, 3])
@pytest.mark.parametrize("pre", ["mirror", "none"])
def test_samples_and_probes_in_one_batch(g, colour_dist, block_width, pre):
    # gmrf_sample_logdet runs the samples and the probes as one block of
    # vectors; every output equals the separate calls bitwise (per-vector
    # arithmetic does not depend on the batch).  Block width 3 makes chunks
    # that straddle the samples / probes boundary.
    shape = (64, 64)
    n = 4096
    k2 = inputs.kappa2_gp_field(shape, seed=1, ell=8.0)
    op = "spde_squared" if pre == "mirror" else "shifted_laplacian"
    with g.Problem(shape, "neumann", op, kappa2=_dev(k2), precond=pre) as p:
        if block_width:
            p.set_tuning(block_width=block_width)
        m_max = 300
        x1 = torch.empty(5 * n, device="cuda")
        rc1, si1 = p.sample(x1, nsamples=5, tol=1e-6, m_max=m_max, seed=11)
        ld1, se1, q1, li1, rc2 = p.logdet(nprobes=4, tol=1e-6, m_max=m_max, seed=12, colour_dist=colour_dist)
        x2 = torch.empty(5 * n, device="cuda")
        rc, si2, ld2, se2, q2, li2 = p.sample_logdet(x2, nsamples=5, nprobes=4, tol=1e-6, m_max=m_max, seed=11,
                                                     probe_seed=12, colour_dist=colour_dist)
        xh = np.zeros((5, n), dtype=np.float32)
        rch, _, ldh, _, _, _ = p.sample_logdet(xh, nsamples=5, nprobes=4, tol=1e-6, m_max=m_max, seed=11,
                                               probe_seed=12, colour_dist=colour_dist)
        with pytest.raises(g.GmrfError):
            p.sample_logdet(x2, nsamples=5, nprobes=4, tol=1e-6, m_max=m_max, seed=11, probe_seed=12,
                            colour_dist=-1)
    # the samples' status is the honest one of gmrf_sample (the unpreconditioned
    # FP32 operator here can stop short of tol); the probes converge
    assert rc == rc1 == rch and rc2 == g.OK
    assert rc1 == g.OK or (pre == "none" and rc1 == g.ERR_NOT_CONVERGED)
    assert torch.equal(x1, x2) and np.array_equal(xh, x1.cpu().numpy().reshape(5, n))
    assert np.array_equal(q1, q2) and ld1 == ld2 == ldh and se1 == se2
    assert [(i.m_used, i.status, i.err_est) for i in si1] == [(i.m_used, i.status, i.err_est) for i in si2]
    assert [i.m_used for i in li1] == [i.m_used for i in li2]
    assert len(q2) == 4 * (colour_dist + 1) ** 2
