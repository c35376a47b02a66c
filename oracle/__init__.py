"""CPU oracle for the matrix-free multilevel deflation Helmholtz solver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 (complex128)
restatement of what the paper computes, used to check the CUDA library.  Only
the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The library never calls it, and it never calls the
library; the two share no code.  The only common dependency is
``model_problems`` (seeded input generators, none of the method's arithmetic).

Modules, each citing the passage it follows:

* ``stencils``   exact Galerkin coarse stencils (Section 3.3, Appendix A).
* ``operators``  A_h, the CSLP M, coarse A_l / M_l with ghost rows
                 (Section 2.1 Eqs. for A_h and the ghost points; Eq. for
                 M_(beta1,beta2); Section 3.3 "Boundary"), and their
                 homogeneous-Dirichlet forms (MP-1a, Section 2.2).
* ``transfers``  deflation Z / Z^T and multigrid full weighting / bilinear
                 (vertex grids and Dirichlet interior-unknown grids).
* ``multigrid``  CSLP approximate inverse by a V-cycle.
* ``krylov``     GMRES / FGMRES with modified Gram-Schmidt (Algorithm 1), and
                 Bi-CGSTAB (van der Vorst 1992) for the CSLP inverse.
* ``madp``       level hierarchy and the recursive deflated FGMRES
                 (Algorithm 1, the MADP schedule of Section 4.4 and the
                 variants of Sections 3.2, 4.3 and 4.5).

Parity status of each function is listed in its module header; functions whose
result is not fixed by an independent pin say "parity unpinned".
"""
