"""CPU FP64 oracle for the Krylov GMRF sampler and the Lanczos log-determinant.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports, calls or links anything here, and this package imports nothing from
the product package: the two share no code.  Inputs that both sides need come
from the seeded generators in ``paper_1312_1476_gb300/inputs.py``, which hold
none of the method's arithmetic.

The oracle is written for a reader checking it against the paper
(Simpson, Turner, Strickland, Pettitt, "Scalable iterative methods for sampling
from massive Gaussian random vectors"):

* ``stencil``  -- the precision matrices Q (Section 2: matrix-free structured Q;
  the library's lattice operators), assembled from Kronecker sums of 1-D graph
  Laplacians, plus a per-cell brute-force assembly used to pin them.
* ``exact``    -- the plain definitions the method converges to: x = Q^{-1/2} z
  (Section 4, principal square root) by dense eigendecomposition or by the
  closed-form spectral transforms of constant-coefficient lattices, and
  log det Q by dense Cholesky or by the closed-form eigenvalues (Section 6).
* ``precond``  -- the constant-coefficient preconditioner M = F F^T of
  Proposition 1 / Theorem 2 (Section 5), applied through its closed-form
  spectrum.
* ``lanczos``  -- Algorithm 1 in FP64 (optionally with full
  reorthogonalisation), the Theorem 1 bounds, the preconditioned sampler of
  Proposition 1, and the Hutchinson / Gauss-quadrature log-determinant of
  Section 6.
* ``sparse``   -- general sparse Q with an incomplete-Cholesky factor F as the
  preconditioner (Section 5.2, Figure 3): the threshold factorisation, and the
  Proposition 1 map x = F^{-T} (F^{-1} Q F^{-T})^{-1/2} z and log-determinant,
  by dense linear algebra.
* ``philox``   -- the Philox-4x32-10 counter-based generator (Salmon et al.,
  SC'11) that the device path uses for z and Rademacher probes, restated from
  its published definition, with the Box-Muller transform.

Parity status of every function is listed in its docstring; a function whose
result is not pinned to something outside the oracle would say "parity
unpinned" (none does: the Philox stream is pinned to an independent
implementation of the generator, the rest to closed forms, dense linear
algebra and brute force; see the tests/test_oracle_*.py files).
"""
