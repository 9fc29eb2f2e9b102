"""GB300-native Krylov (Lanczos) sampler and log-determinant for lattice GMRFs.

Simpson, Turner, Strickland, Pettitt, "Scalable iterative methods for sampling
from massive Gaussian random vectors": Algorithm 1 (Section 4), the
preconditioned sampler of Proposition 1 with the circulant preconditioner of
Section 5.1, and the Hutchinson / Lanczos-quadrature log det of Section 6.

The compute path is the C-ABI CUDA library ``libgmrf.so`` (include/gmrf.h);
``paper_1312_1476_gb300.gmrf`` is its Python binding.  Importing this package
loads nothing; ``from paper_1312_1476_gb300 import gmrf`` loads the library
and raises if it has not been built.
"""
