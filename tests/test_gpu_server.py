"""GPU tests of the continuous-batching server (gmrf_server_*): requests whose
vectors share the slot table, admitted as slots free up, some while others
are in mid-iteration, give bitwise the results of the synchronous calls
(gmrf_sample / gmrf_logdet on a problem with the request's tau); log-det
requests larger than the slot table are admitted a part at a time; while a
server exists its problem refuses other calls."""
import numpy as np
import pytest

from paper_1312_1476_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    from paper_1312_1476_gb300 import gmrf
    assert torch.cuda.is_available()
    return gmrf


CASES = [((64, 64), "neumann", "spde_squared", "mirror", "fp32"),
         ((32, 64), "neumann", "spde_squared", "circulant", "fp32"),
         ((24, 20, 16), "dirichlet", "shifted_laplacian", "none", "fp32"),
         ((48, 40), "dirichlet", "shifted_laplacian", "none", "fp64")]

TOL = {"fp32": 1e-6, "fp64": 1e-10}


def _problem(g, shape, bc, op, pre, precision, tau):
    k2 = inputs.kappa2_gp_field(shape, seed=5, ell=6.0) if len(shape) == 2 else \
        inputs.kappa2_uniform_field(shape, seed=5, lo=0.05, hi=1.0)
    return g.Problem(shape, bc, op, kappa2=torch.from_numpy(k2).cuda(), tau=tau, precond=pre, precision=precision)


@pytest.mark.parametrize("shape,bc,op,pre,precision", CASES)
def test_server_equals_synchronous_calls(g, shape, bc, op, pre, precision):
    n = int(np.prod(shape))
    dt = torch.float64 if precision == "fp64" else torch.float32
    tol, m_max, ce = TOL[precision], 600, 8
    # (kind, count, seed, tau); the second group arrives while the first runs
    first = [("sample", 3, 11, 1.0), ("logdet", 9, 12, 2.5), ("sample", 1, 13, 0.7)]
    later = [("sample", 5, 14, 3.0), ("logdet", 4, 15, 1.0), ("sample", 2, 16, 4.5)]
    out = {}
    with _problem(g, shape, bc, op, pre, precision, 1.0) as p:
        with g.Server(p, nslots=6, m_max=m_max, tol=tol, check_every=ce) as sv:
            ids = []

            def submit(reqs):
                for kind, cnt, seed, tau in reqs:
                    if kind == "sample":
                        x = torch.full((cnt * n,), float("nan"), dtype=dt, device="cuda")
                        ids.append((sv.submit_sample(x, cnt, seed, tau), kind, cnt, seed, tau, x))
                    else:
                        ids.append((sv.submit_logdet(cnt, seed, tau), kind, cnt, seed, tau, None))

            submit(first)
            sv.step()
            sv.step()
            submit(later)
            # while the server exists the problem serves it alone
            xx = torch.empty(n, dtype=dt, device="cuda")
            rc, _ = p.sample(xx, nsamples=1, tol=tol, m_max=m_max, seed=1, raise_on_error=False)
            assert rc == g.ERR_INVALID
            for _ in range(10000):
                if sv.step() == 0:
                    break
            assert sv.step() == 0
            for rid, kind, cnt, seed, tau, x in ids:
                res = sv.poll(rid)
                assert res is not None
                out[rid] = (kind, cnt, seed, tau, x, res)
    for rid, (kind, cnt, seed, tau, x, (rc, infos, ld, se)) in out.items():
        with _problem(g, shape, bc, op, pre, precision, tau) as p1:
            if kind == "sample":
                x1 = torch.empty(cnt * n, dtype=dt, device="cuda")
                rc1, i1 = p1.sample(x1, nsamples=cnt, tol=tol, m_max=m_max, seed=seed, check_every=ce,
                                    raise_on_error=False)
                assert torch.equal(x, x1)
            else:
                ld1, se1, _, i1, rc1 = p1.logdet(nprobes=cnt, tol=tol, m_max=m_max, seed=seed, check_every=ce,
                                                 raise_on_error=False)
                assert ld == ld1 and (se == se1 or (np.isnan(se) and np.isnan(se1)))
        assert rc == rc1
        assert [(a.m_used, a.status, a.err_est) for a in infos] == [(b.m_used, b.status, b.err_est) for b in i1]


def test_server_rejects_bad_requests(g):
    with _problem(g, (32, 32), "neumann", "spde_squared", "mirror", "fp32", 1.0) as p:
        with pytest.raises(g.GmrfError):
            g.Server(p, nslots=0)
        with g.Server(p, nslots=2, m_max=50) as sv:
            host = np.zeros(1024, dtype=np.float32)
            with pytest.raises(g.GmrfError):
                sv.submit_sample(host, 1, 1)  # host output
            with pytest.raises(g.GmrfError):
                sv.submit_logdet(0, 1)
            with pytest.raises(g.GmrfError):
                sv.submit_logdet(4, 1, tau=-1.0)
            with pytest.raises(g.GmrfError):
                g.Server(p, nslots=2)  # one server per problem
            assert sv.step() == 0
        # after the server is gone the problem takes calls again
        x = torch.empty(1024, dtype=torch.float32, device="cuda")
        rc, _ = p.sample(x, nsamples=1, tol=1e-6, m_max=200, seed=1)
        assert rc == g.OK


@pytest.mark.parametrize("precision,with_factor", [("fp64", True), ("fp64", False), ("fp32", True)])
def test_server_sparse_equals_synchronous_calls(g, precision, with_factor):
    # the slot server on a CSR precision with an incomplete-Cholesky factor
    # (Section 5.2): samples (x = F^{-T} A^{-1/2} z) and log dets bitwise equal
    # to gmrf_sample / gmrf_logdet on a problem with the request's tau
    Q = inputs.figure3_matrix()
    F = g.ichol(Q, droptol=1e-3, shift=1e-3) if with_factor else None
    n = Q[0].shape[0] - 1 if isinstance(Q, tuple) else Q.shape[0]
    dt = torch.float64 if precision == "fp64" else torch.float32
    tol = TOL[precision]
    reqs = [("sample", 3, 21, 1.0), ("logdet", 5, 22, 2.0), ("sample", 2, 23, 0.5)]
    out = {}
    with g.SparseProblem(Q, F, tau=1.0, precision=precision) as p:
        with g.Server(p, nslots=4, m_max=800, tol=tol, check_every=8) as sv:
            ids = []
            for kind, cnt, seed, tau in reqs:
                if kind == "sample":
                    x = torch.full((cnt * n,), float("nan"), dtype=dt, device="cuda")
                    ids.append((sv.submit_sample(x, cnt, seed, tau), kind, cnt, seed, tau, x))
                else:
                    ids.append((sv.submit_logdet(cnt, seed, tau), kind, cnt, seed, tau, None))
            for _ in range(10000):
                if sv.step() == 0:
                    break
            for rid, kind, cnt, seed, tau, x in ids:
                out[rid] = (kind, cnt, seed, tau, x, sv.poll(rid))
    for rid, (kind, cnt, seed, tau, x, (rc, infos, ld, se)) in out.items():
        with g.SparseProblem(Q, F, tau=tau, precision=precision) as p1:
            if kind == "sample":
                x1 = torch.empty(cnt * n, dtype=dt, device="cuda")
                rc1, i1 = p1.sample(x1, nsamples=cnt, tol=tol, m_max=800, seed=seed, check_every=8,
                                    raise_on_error=False)
                assert torch.equal(x, x1)
            else:
                ld1, se1, _, i1, rc1 = p1.logdet(nprobes=cnt, tol=tol, m_max=800, seed=seed, check_every=8,
                                                 raise_on_error=False)
                assert ld == ld1 and (se == se1 or (np.isnan(se) and np.isnan(se1)))
        assert rc == rc1
        assert [(a.m_used, a.status, a.err_est) for a in infos] == [(b.m_used, b.status, b.err_est) for b in i1]


def test_server_smmala_operator_equals_synchronous_calls(g):
    # the sMMALA operator tau((kc^2 + L)^2 + D) preconditioned by its prior (circulant on a torus)
    shape = (64, 64)
    n = 64 * 64
    d = inputs.kappa2_uniform_field(shape, seed=8, lo=0.0, hi=3.0)
    kw = dict(kappa2=torch.from_numpy(d).cuda(), kappa2_const=0.5, precond="circulant", precision="fp32")
    reqs = [("sample", 3, 31, 1.0), ("logdet", 6, 32, 2.0), ("sample", 4, 33, 0.8)]
    out = {}
    with g.Problem(shape, "periodic", "spde_plus_diag", tau=1.0, **kw) as p:
        with g.Server(p, nslots=5, m_max=300, tol=1e-6, check_every=8) as sv:
            ids = []
            for kind, cnt, seed, tau in reqs:
                if kind == "sample":
                    x = torch.full((cnt * n,), float("nan"), dtype=torch.float32, device="cuda")
                    ids.append((sv.submit_sample(x, cnt, seed, tau), kind, cnt, seed, tau, x))
                else:
                    ids.append((sv.submit_logdet(cnt, seed, tau), kind, cnt, seed, tau, None))
            for _ in range(10000):
                if sv.step() == 0:
                    break
            for rid, kind, cnt, seed, tau, x in ids:
                out[rid] = (kind, cnt, seed, tau, x, sv.poll(rid))
    for rid, (kind, cnt, seed, tau, x, (rc, infos, ld, se)) in out.items():
        with g.Problem(shape, "periodic", "spde_plus_diag", tau=tau, **kw) as p1:
            if kind == "sample":
                x1 = torch.empty(cnt * n, dtype=torch.float32, device="cuda")
                rc1, i1 = p1.sample(x1, nsamples=cnt, tol=1e-6, m_max=300, seed=seed, check_every=8,
                                    raise_on_error=False)
                assert torch.equal(x, x1)
            else:
                ld1, se1, _, i1, rc1 = p1.logdet(nprobes=cnt, tol=1e-6, m_max=300, seed=seed, check_every=8,
                                                 raise_on_error=False)
                assert ld == ld1 and se == se1
        assert rc == rc1 == g.OK
        assert [(a.m_used, a.status, a.err_est) for a in infos] == [(b.m_used, b.status, b.err_est) for b in i1]
