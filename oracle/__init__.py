"""CPU FP64 oracle for the matrix-free P1/P2 hot path (test infrastructure).

This package is test infrastructure only: the tests, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product library never
does, and it imports nothing from the product.  It is plain, slow, obviously
correct NumPy/SciPy written from the paper (Kohl, Bauer, Boehm, Ruede,
"Fundamental data structures for matrix-free finite elements on hybrid
tetrahedral grids"):

* ``indexing``  - polytope index sets, cardinalities and the linearisation
                  t_w of Sec. 4 (the tetrahedral-number and linearisation equations and the AoS/SoA forms).
* ``mesh``      - Bey's regular refinement (Sec. 3.1, eight-children rule) applied recursively to
                  every macro cell, plus an independent lattice enumeration of
                  the six micro-cell subgroups (Sec. 3.2, Table 1).
* ``fem``       - textbook P1/P2 element matrices and COO->CSR assembly of the
                  global matrix (Sec. 5.2, element-wise sum).
* ``quadrature``- the fixed quadrature rules used by the variable-coefficient
                  P2 operator and an error-bound rule.
* ``gmg``       - textbook geometric multigrid on the assembled matrices
                  (Jacobi, colour-ordered Gauss-Seidel, Chebyshev, FMG).
* ``nedelec``   - lowest-order Nedelec elements for the curl-curl problem of
                  Sec. 6: Whitney basis, transfers, discrete gradient and
                  Hiptmair multigrid.
* ``surrogate`` - polynomial surrogate stencils of the variable-coefficient P1
                  operator (Sec. 5.2, surrogates).
* ``mlp``       - FP64 forward/backward of the local learned smoother network.

Parity status of each function is stated in its module docstring.
"""
