"""GPU test of gmrf_apply_inv_sqrt_noalloc, the allocation-free variant of
gmrf_apply(which = 2) for callers that must not allocate device memory during
the call (an application that routes all device memory through its own pool,
or a latency-critical loop).  Its output must equal the allocating entry
point's, on two calls in a row that share the library's static scratch array.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1312_1476_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    from paper_1312_1476_gb300 import _build
    _build.build()
    from paper_1312_1476_gb300 import gmrf
    assert torch.cuda.is_available()
    return gmrf


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [((1024, 1024), "neumann", "mirror", "fp32", 3, 3e-6),
         ((256, 128), "neumann", "circulant", "fp32", 5, 3e-6),
         ((16, 32), "dirichlet", "circulant", "fp64", 2, 1e-12),
         ((64, 64), "periodic", "mirror", "fp64", 4, 1e-12)]


@pytest.mark.parametrize("shape,bc,kind,precision,nvec,tol", CASES)
def test_noalloc_matches_apply_twice(g, shape, bc, kind, precision, nvec, tol):
    n = int(np.prod(shape))
    k2 = torch.from_numpy(inputs.kappa2_gp_field(shape, seed=1, ell=8.0)).cuda()
    dt = torch.float64 if precision == "fp64" else torch.float32
    with g.Problem(shape, bc, "spde_squared", kappa2=k2, tau=1.7, precond=kind, precision=precision) as p:
        y_ref = torch.empty(nvec * n, dtype=dt, device="cuda")
        y_na = torch.empty(nvec * n, dtype=dt, device="cuda")
        for call in range(2):
            v = torch.from_numpy(inputs.gaussian_vectors(nvec, n, seed=10 + call).reshape(-1)).to(dt).cuda()
            p.apply(2, v, y_ref, nvec=nvec)
            y_na.fill_(float("nan"))
            p.apply_inv_sqrt_noalloc(v, y_na, nvec=nvec)
            torch.cuda.synchronize()
            assert torch.isfinite(y_na).all()
            assert _rel(y_na, y_ref) <= tol


def test_noalloc_rejects_what_it_cannot_serve(g):
    n = 1024 * 1024
    with g.Problem((1024, 1024), "neumann", "spde_squared", kappa2_const=0.05, precond="mirror") as p:
        # 8 vectors of a 1024^2 FP32 grid need more than the 32 MiB scratch
        v = torch.zeros(8 * n, dtype=torch.float32, device="cuda")
        y = torch.zeros(8 * n, dtype=torch.float32, device="cuda")
        rc = g.lib().gmrf_apply_inv_sqrt_noalloc(p._h, 8, ctypes.c_void_p(v.data_ptr()),
                                                 ctypes.c_void_p(y.data_ptr()))
        assert rc == g.ERR_INVALID
        # host buffers are rejected (no staging copies)
        vh = np.zeros(n, dtype=np.float32)
        yh = np.zeros(n, dtype=np.float32)
        rc = g.lib().gmrf_apply_inv_sqrt_noalloc(p._h, 1, ctypes.c_void_p(vh.ctypes.data),
                                                 ctypes.c_void_p(yh.ctypes.data))
        assert rc == g.ERR_INVALID
    with g.Problem((32, 32), "neumann", "spde_squared", kappa2_const=0.05) as p:
        v = torch.zeros(1024, dtype=torch.float32, device="cuda")
        rc = g.lib().gmrf_apply_inv_sqrt_noalloc(p._h, 1, ctypes.c_void_p(v.data_ptr()),
                                                 ctypes.c_void_p(v.data_ptr()))
        assert rc == g.ERR_INVALID  # no preconditioner
