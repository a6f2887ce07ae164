"""FP64 CPU oracle for the SFFT hot path (arXiv:2109.09334).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The GPU library and
its Python binding never import it, and it imports nothing from them.

Three independent tiers:

* ``liboracle.so`` (``sfft_oracle.c``): the lag-sum form of App. B
  (Eq. B5-B16) with every lag value a direct circular spatial sum, a
  hand-written Cholesky solve, and the literal circular subtraction of Eq. 12;
  polynomial (Eq. 2, 6) or tensor-product B-spline (Eq. 7-9) variation, the
  B-splines by its own Cox-de Boor recursion.
* :mod:`oracle.bruteforce`: the least-squares definition written out -- an
  explicit design matrix ``C`` (one column per unknown, Eq. 11-12), ``M = C^T C``,
  ``rhs = C^T S`` and a library least-squares solve.  Tiny images only.
* :mod:`oracle.decorr`: the noise decorrelation filter of App. C (Eq. 24) for one
  pair, with numpy's FFT as the DFT primitive.
* :mod:`oracle.fourier`: Eq. 19-24 evaluated literally as frequency sums of
  spectrum products with the basis spectra of Eq. 14 (numpy FFT as the DFT
  primitive).  Tiny images only.

Function by function, the pins (in ``tests/test_oracle_*.py``) are: brute
force on tiny images, the closed-form w=0 regression, the one-pixel shift,
exact recovery of an injected kernel, symmetry and positive semidefiniteness,
structural zeros, Toeplitz structure, flux conservation, the residual-energy
identity and the Parseval link between the Fourier and real-space forms; for
the B-spline bases (``tests/test_oracle_bspline.py``) scipy's B-splines,
partition of unity, the brute-force design matrix on scipy's basis, the
degree-0 reduction to the constant polynomial, exact recovery and the
constant-ratio kernel sum.  The frequency-domain tier covers the polynomial
basis only (the basis does not enter the Fourier reading it pins).
"""
from .core import (  # noqa: F401
    OracleConfig,
    bspline,
    build_system,
    cholesky_solve,
    decode_unknown,
    lag_sum,
    library_path,
    num_unknowns,
    subtract,
    subtract_pixels,
    system_entries,
    threads,
)
