"""Cross-check of the library's FFT/DCT preconditioner (Section 5.1) against
cuFFT through torch.fft, on the GPU: y = M^{-1/2} v with M = tau (kbar^2 + L)^p
on the torus (circulant, 2-D FFT) and on the cell-centred Neumann grid
(mirror, the 2-D FFT of the even extension to 2N x 2N).  cuFFT is a cross-check
only; the parity reference of the library is the CPU oracle."""
import math

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


def _lam(N, period):
    k = torch.arange(period, dtype=torch.float64, device="cuda")
    return 2.0 - 2.0 * torch.cos(2.0 * math.pi * k / period)


def _cufft_inv_sqrt(v, ny, nx, kind, kbar2, tau, power):
    """M^{-1/2} v in FP64 with torch.fft (cuFFT); v is [ny][nx]."""
    if kind == "circulant":
        mu = tau * (kbar2 + _lam(ny, ny)[:, None] + _lam(nx, nx)[None, :]) ** power
        return torch.fft.ifft2(torch.fft.fft2(v) / torch.sqrt(mu)).real
    # even extension: x~[2N-1-i] = x[i] in each direction; the Neumann operator's
    # eigenvalues are those of the 2N-periodic Laplacian
    ext = torch.cat([v, torch.flip(v, [0])], 0)
    ext = torch.cat([ext, torch.flip(ext, [1])], 1)
    mu = tau * (kbar2 + _lam(ny, 2 * ny)[:, None] + _lam(nx, 2 * nx)[None, :]) ** power
    return torch.fft.ifft2(torch.fft.fft2(ext) / torch.sqrt(mu)).real[:ny, :nx]


@pytest.mark.parametrize("shape,kind,bc", [((1024, 1024), "mirror", "neumann"), ((512, 1024), "circulant", "periodic"),
                                           ((256, 2048), "mirror", "neumann"), ((128, 128), "circulant", "periodic")])
@pytest.mark.parametrize("op,power", [("spde_squared", 2), ("shifted_laplacian", 1)])
def test_inv_sqrt_against_cufft(g, shape, kind, bc, op, power):
    ny, nx = shape
    n = nx * ny
    kb, tau = 0.05, 2.5
    V = inputs.gaussian_vectors(2, n, seed=17, dtype=np.float32)
    with g.Problem(shape, bc, op, kappa2_const=0.3, tau=tau, precond=kind, kappa2_precond=kb) as p:
        y = torch.empty(2 * n, dtype=torch.float32, device="cuda")
        p.apply(2, torch.from_numpy(V).cuda(), y, nvec=2)
    for s in range(2):
        v = torch.from_numpy(V[s].astype(np.float64)).cuda().reshape(ny, nx)
        ref = _cufft_inv_sqrt(v, ny, nx, kind, kb, tau, power)
        err = float(torch.linalg.vector_norm(y[s * n:(s + 1) * n].double().reshape(ny, nx) - ref) /
                    torch.linalg.vector_norm(ref))
        assert err <= 3e-6, (shape, kind, op, err)
