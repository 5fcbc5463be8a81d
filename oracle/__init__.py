"""CPU oracle for the space-time KKT method of Deng, Cai and Zou (arXiv 1508.06103).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 CPU statement
of what the method computes, written from the paper.  Only the tests, the
smoke check and the CPU-baseline leg of the benchmark may import it; the
library's product path never does, and it shares no code with the CUDA path
(the only common module is the seeded input generator, which holds none of
the method's arithmetic).

Modules
-------
fem       Q1 element matrices by quadrature and global assembly of the
          spatial matrices B, A, E, K and the 1D time matrices (Appendix).
kkt       The all-at-once KKT matrix F_h in point-block order, its right-hand
          side, a level-by-level matvec, and source extraction (Sec. 3.1-3.2,
          Appendix).
forward   Forward (state) and backward (adjoint) time marching (Eq. 8) used to
          make observation data (Sec. 4) and the reduced-space solve.
schwarz   Space-time subdomains, ILU(0)/LU subdomain solves, one-level RAS,
          nested interpolation/restriction and the two-level hybrid (Sec. 3.2).
krylov    Restarted right-preconditioned GMRES and flexible GMRES (Sec. 3.2, 4).

Parity status of each function is stated in its module header; every
function is pinned by a CPU test unless its header says "parity unpinned".
"""
