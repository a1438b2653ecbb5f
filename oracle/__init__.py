"""CPU oracle for the 2-level DD-alpha-AMG Wilson-clover hot path (TEST INFRASTRUCTURE).

This package is a plain, slow, FP64 restatement (PyTorch CPU tensors,
complex128) of what the paper's method computes, written to check the CUDA
library against.  It is test
infrastructure only: the tests, the smoke check and the benchmark's CPU
baseline leg may import it; the library never does, and it shares no code,
tables or constants with the CUDA path.

Modules follow the paper's structure (arXiv 1811.00355, "Porting DDalphaAMG
solver to K computer", Sec. 2 "Algorithm" and Sec. 3):

* :mod:`oracle.lattice`  index maps: sites, parities, Schwarz blocks,
  aggregates, coarse lattice (Sec. 2, Fig. 1);
* :mod:`oracle.dirac`    gamma matrices, clover term, Wilson-clover D, packed
  Hermitian clover blocks (Sec. 1, Sec. 3);
* :mod:`oracle.sap`      site even-odd MR block solver and multiplicative SAP
  smoother (Sec. 2);
* :mod:`oracle.coarse`   test-vector orthonormalisation, restriction R and
  prolongation P (Eq. 3, Eq. 4), coarse operator (Eq. 2), coarse stencil and
  even-odd GMRES (Sec. 2);
* :mod:`oracle.solver`   preconditioner M (Eq. 5), outer flexible GMRES,
  adaptive setup (Sec. 2);
* :mod:`oracle.three_level`  the same construction applied once more to
  D_c (the recursion Sec. 1 names as a merit, not run in the paper): level-2
  Schwarz smoother, aggregation, D_cc = P2^H D_c P2, and the three-level M;
* :mod:`oracle.critical_mass`  the smallest singular value of D and the most
  critical bare mass of a gauge field on a proxy lattice (a workload
  parameter, not a step of the method).

Every function that is checked only by the invariants it must satisfy, and
not against an independent value, says so.  The adaptive setup's output is
"parity unpinned" as a unique result (it depends on rounding); it is pinned
only through the invariants P^H P = 1 and D_c = P^H D P.  The same holds for
the level-2 setup of the three-level method (P2^H P2 = 1, D_cc = P2^H D_c P2).
"""
