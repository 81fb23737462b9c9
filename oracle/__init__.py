"""Plain, slow, CPU FP64 oracle for the SCSF hot path (test infrastructure).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it. The GPU product path
never imports, links or calls anything here, and nothing here imports the
GPU package: the two share no code. The only shared module is
``scsf_inputs`` (seeded workload definitions, no method arithmetic).

Contents (paper: "Accelerating Eigenvalue Dataset Generation via Chebyshev
Subspace Filter"):

* ``operators``  - FDM assembly of -div(a grad u) and -Lap u + V u (Sec. 2.1,
  Eq. (eq_p) and App. D.2), Gershgorin bounds, relative residual (App. D.5).
* ``sort``       - truncated-DFT features and the greedy chain (Alg. 2).
* ``chebyshev``  - Chebyshev polynomials (Sec. 2.2) and the scaled filter
  (Alg. 1).
* ``chfsi``      - Chebyshev filtered subspace iteration with Householder QR
  (Alg. 3) and the warm-started chain over a sorted sequence (Sec. 3.2).
* ``dense``      - the plain definition of the k smallest eigenpairs (dense
  symmetric eigensolve) and a textbook cyclic Jacobi for tiny matrices.
* ``sturm``      - 1-D tridiagonal Sturm bisection and closed forms used to
  pin the rest (App. C and the separable special cases).
* ``inertia``    - Sylvester inertia count via banded LDL^T.
* ``compare``    - eigenvalue / eigenspace comparisons used by tests.
* ``products``   - correctly rounded block products A^T B and X M (the Gram,
  Rayleigh-Ritz and rotation products of Alg. 3), for the tensor-core products.

Every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, worked examples and brute force, none of which reuse the function's
own formula.
"""
from . import operators, sort, chebyshev, chfsi, dense, sturm, inertia, compare, products  # noqa: F401
