"""GPU parity of the building blocks against the oracle: the Philox streams,
the matrix-free stencil apply Q v (Section 2), and the fast preconditioner
apply M^{-1/2} v and preconditioned operator A v (Proposition 1)."""
import numpy as np
import pytest

from oracle import lanczos as olz
from oracle import philox, precond, stencil
from paper_1312_1476_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    from paper_1312_1476_gb300 import gmrf
    assert torch.cuda.is_available()
    return gmrf


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def test_rng_words_bitexact(g):
    nvec, n, seed = 3, 1001, 0x1234_5678_9ABC
    out = torch.empty(nvec * 4 * ((n + 3) // 4), dtype=torch.int32, device="cuda")
    g.rng(2, nvec, n, seed, out)
    w = out.cpu().numpy().view(np.uint32).reshape(nvec, -1)
    np.testing.assert_array_equal(w, philox.gaussian_words(nvec, n, seed))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_rng_gaussian_and_rademacher(g, precision):
    nvec, n, seed = 4, 4099, 77
    dt = torch.float64 if precision == "fp64" else torch.float32
    z = torch.empty(nvec * n, dtype=dt, device="cuda")
    g.rng(0, nvec, n, seed, z, precision=precision)
    ref = philox.gaussian(nvec, n, seed)
    tol = 1e-12 if precision == "fp64" else 2e-5
    assert np.abs(z.cpu().numpy().reshape(nvec, n) - ref).max() <= tol
    r = torch.empty(nvec * n, dtype=dt, device="cuda")
    g.rng(1, nvec, n, seed, r, precision=precision)
    np.testing.assert_array_equal(r.cpu().numpy().reshape(nvec, n), philox.rademacher(nvec, n, seed))


STENCIL_CASES = [((17, 23), "periodic", "shifted_laplacian"), ((17, 23), "neumann", "shifted_laplacian"),
                 ((17, 23), "dirichlet", "shifted_laplacian"), ((33, 20), "periodic", "spde_squared"),
                 ((33, 20), "neumann", "spde_squared"), ((33, 20), "dirichlet", "spde_squared"),
                 ((5, 7, 9), "periodic", "shifted_laplacian"), ((5, 7, 9), "neumann", "shifted_laplacian"),
                 ((9, 40, 35), "dirichlet", "shifted_laplacian"), ((3, 2, 70), "periodic", "shifted_laplacian"),
                 ((4, 9, 128), "dirichlet", "shifted_laplacian"), ((5, 6, 256), "periodic", "shifted_laplacian"),
                 ((3, 17, 132), "neumann", "shifted_laplacian"), ((19, 3, 64), "periodic", "shifted_laplacian"),
                 ((70, 12, 384), "neumann", "shifted_laplacian"), ((37, 29, 256), "dirichlet", "shifted_laplacian"),
                 # 2-D grids streamed in strips of 128 (FP32) / 64 (FP64) columns: one or several strips,
                 # row counts that leave partial slabs and partial row chunks
                 ((513, 128), "periodic", "shifted_laplacian"), ((256, 512), "neumann", "shifted_laplacian"),
                 ((1030, 128), "dirichlet", "shifted_laplacian"), ((256, 256), "periodic", "spde_squared"),
                 ((300, 256), "neumann", "spde_squared"), ((260, 384), "dirichlet", "spde_squared")]


@pytest.mark.parametrize("shape,bc,op", STENCIL_CASES)
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_stencil_apply(g, shape, bc, op, precision):
    n = int(np.prod(shape))
    k2 = inputs.kappa2_uniform_field(shape, seed=4, lo=0.05, hi=1.0)
    Q = stencil.precision_matrix(shape, bc, op, k2.astype(np.float64), tau=1.7)
    dt = np.float64 if precision == "fp64" else np.float32
    V = inputs.gaussian_vectors(3, n, seed=5, dtype=dt)
    with g.Problem(shape, bc, op, kappa2=_dev(k2), tau=1.7, precision=precision) as p:
        y = torch.empty(3 * n, dtype=torch.float64 if precision == "fp64" else torch.float32, device="cuda")
        p.apply(0, _dev(V), y, nvec=3)
        Y = y.cpu().numpy().reshape(3, n)
    for s in range(3):
        ref = Q @ V[s].astype(np.float64)
        assert _rel(Y[s], ref) <= (1e-13 if precision == "fp64" else 2e-6)


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_stencil_apply_3d_constant_kappa(g, bc):
    # 3-D 7-point apply with a constant coefficient (no kappa^2 field), several
    # z chunks and a ragged tile in y
    shape = (66, 10, 128)
    n = int(np.prod(shape))
    Q = stencil.precision_matrix(shape, bc, "shifted_laplacian", 0.37, tau=1.3)
    V = inputs.gaussian_vectors(2, n, seed=12, dtype=np.float32)
    with g.Problem(shape, bc, "shifted_laplacian", kappa2_const=0.37, tau=1.3) as p:
        y = torch.empty(2 * n, dtype=torch.float32, device="cuda")
        p.apply(0, _dev(V), y, nvec=2)
        Y = y.cpu().numpy().reshape(2, n)
    for s in range(2):
        assert _rel(Y[s], Q @ V[s].astype(np.float64)) <= 2e-6


PRE_CASES = [((8, 8), "periodic"), ((16, 32), "periodic"), ((64, 64), "neumann"), ((32, 16), "neumann"),
             ((256, 256), "periodic"), ((256, 128), "neumann"), ((1024, 1024), "neumann"),
             ((1024, 1024), "periodic")]


@pytest.mark.parametrize("shape,kind", PRE_CASES)
@pytest.mark.parametrize("op", ["shifted_laplacian", "spde_squared"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_precond_inv_sqrt(g, shape, kind, op, precision):
    n = int(np.prod(shape))
    dt = np.float64 if precision == "fp64" else np.float32
    V = inputs.gaussian_vectors(2, n, seed=6, dtype=dt)
    kb = 0.05
    gk = "circulant" if kind == "periodic" else "mirror"
    with g.Problem(shape, "neumann", op, kappa2_const=0.3, tau=2.5, precond=gk, kappa2_precond=kb,
                   precision=precision) as p:
        y = torch.empty(2 * n, dtype=torch.from_numpy(V).dtype, device="cuda")
        p.apply(2, _dev(V), y, nvec=2)
        Y = y.cpu().numpy().reshape(2, n)
    for s in range(2):
        ref = precond.apply_power(shape, kind, op, kb, 2.5, V[s].astype(np.float64), -0.5)
        assert _rel(Y[s], ref) <= (1e-12 if precision == "fp64" else 3e-6)


OPER_CASES = [((16, 16), "neumann", "periodic"), ((16, 16), "dirichlet", "periodic"),
              ((16, 16), "periodic", "periodic"), ((32, 16), "neumann", "neumann"),
              ((16, 32), "dirichlet", "neumann"), ((16, 16), "periodic", "neumann"),
              ((128, 128), "neumann", "periodic"), ((128, 128), "neumann", "neumann"),
              ((1024, 1024), "neumann", "neumann"), ((512, 1024), "dirichlet", "periodic"),
              ((1024, 512), "periodic", "neumann"),
              # several row blocks with y-boundary terms of R (generic path: w rows across blocks)
              ((64, 32), "dirichlet", "periodic"), ((64, 32), "neumann", "periodic"),
              ((128, 32), "dirichlet", "neumann")]


@pytest.mark.parametrize("shape,bc,kind", OPER_CASES)
@pytest.mark.parametrize("op", ["shifted_laplacian", "spde_squared"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_preconditioned_operator(g, shape, bc, kind, op, precision):
    n = int(np.prod(shape))
    k2 = inputs.kappa2_gp_field(shape, seed=1, ell=shape[0] / 16.0)
    kb = precond.kappa2_bar(k2)
    Q = stencil.precision_matrix(shape, bc, op, k2.astype(np.float64), tau=3.0)
    A = olz.preconditioned_operator(Q, shape, kind, op, kb, 3.0)
    dt = np.float64 if precision == "fp64" else np.float32
    V = inputs.gaussian_vectors(2, n, seed=8, dtype=dt)
    gk = "circulant" if kind == "periodic" else "mirror"
    with g.Problem(shape, bc, op, kappa2=_dev(k2), tau=3.0, precond=gk, kappa2_precond=kb,
                   precision=precision) as p:
        y = torch.empty(2 * n, dtype=torch.from_numpy(V).dtype, device="cuda")
        p.apply(1, _dev(V), y, nvec=2)
        Y = y.cpu().numpy().reshape(2, n)
    for s in range(2):
        ref = A(V[s].astype(np.float64))
        assert _rel(Y[s], ref) <= (1e-12 if precision == "fp64" else 3e-6)



@pytest.mark.parametrize("bc", ["periodic", "neumann", "dirichlet"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_stencil_strip_plus_diag_and_constant_kappa(g, bc, precision):
    # the streamed 2-D kernel on Q = tau((kc + L)^2 + D) and on a constant-kappa^2
    # squared operator (the coefficient taken in the problem's precision)
    shape = (264, 256)
    n = 264 * 256
    d = inputs.kappa2_uniform_field(shape, seed=6, lo=0.2, hi=2.0)
    dt = np.float64 if precision == "fp64" else np.float32
    V = inputs.gaussian_vectors(2, n, seed=7, dtype=dt)
    tol = 1e-13 if precision == "fp64" else 2e-6
    Q = stencil.precision_matrix(shape, bc, "spde_plus_diag", d.astype(np.float64), 1.3, kappa2_prior=0.37)
    with g.Problem(shape, bc, "spde_plus_diag", kappa2=_dev(d), kappa2_const=0.37, tau=1.3,
                   precision=precision) as p:
        y = torch.empty(2 * n, dtype=torch.from_numpy(V).dtype, device="cuda")
        p.apply(0, _dev(V), y, nvec=2)
        Y = y.cpu().numpy().reshape(2, n)
    for s_ in range(2):
        assert _rel(Y[s_], Q @ V[s_].astype(np.float64)) <= tol
    kc = 0.1234567890123
    Q2 = stencil.precision_matrix(shape, bc, "spde_squared", kc, 0.9)
    with g.Problem(shape, bc, "spde_squared", kappa2_const=kc, tau=0.9, precision=precision) as p:
        y = torch.empty(2 * n, dtype=torch.from_numpy(V).dtype, device="cuda")
        p.apply(0, _dev(V), y, nvec=2)
        Y = y.cpu().numpy().reshape(2, n)
    for s_ in range(2):
        assert _rel(Y[s_], Q2 @ V[s_].astype(np.float64)) <= tol
