"""Plain FP64 CPU oracle for the high-order multigrid solvers of Sundar, Stadler & Biros,
"Comparison of multigrid algorithms for high-order continuous finite element
discretizations" (arXiv:1402.5938).

TEST INFRASTRUCTURE ONLY. Nothing in the library's product path may import or run
this package: only the test-suite, the smoke check and the benchmark's CPU-baseline
leg use it. It shares no code, tables or constants with the CUDA library.

The oracle assembles sparse matrices from their definitions (the paper's own
prototype also used assembled operators, Sec. 2.3) and runs the iterations step
by step in the order the paper states them:

* ``basis``     -- GLL nodes, Gauss rule, Lagrange basis (Sec. 2.3, Fig. 1)
* ``fem``       -- mapped mesh, isoparametric geometry, stiffness/mass assembly,
                   Dirichlet elimination (Sec. 2.1 Eq. for A_k, M_k, f_k; Sec. 2.3)
* ``transfer``  -- prolongation P_ij = phi_j^{k-1}(p_i) and R = P^T (Sec. 2.2, Eq. Pstencil)
* ``multigrid`` -- Jacobi / Chebyshev-Jacobi smoothers, Arnoldi eigenvalue estimate,
                   h/p hierarchies, V-cycle, MG as solver, MG-preconditioned CG
                   (Sec. 3.1, 3.2, 4.3, Algorithm 1)

Every function is pinned by tests in ``tests/test_oracle_*.py`` against closed forms,
textbook special cases, invariants, brute force and the iteration counts of the
paper's Tables 1 and 4.
"""
