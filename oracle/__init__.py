"""CPU oracle for the two-level Schwarz / H_k-GenEO / FGMRES Helmholtz solver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
arXiv 2406.06283 (Schwarz preconditioner with the H_k-GenEO coarse space for
indefinite Helmholtz) written with numpy/scipy, used to check the CUDA
library.  Only the test-suite, the smoke check and the CPU-baseline leg of the
benchmark may import it; the library never calls it and shares no code with
it (the two only receive the same seeded inputs).

Modules, each citing the passages it follows:
  fem            P1 Galerkin matrices B, A (stiffness), S (mass), D_k (Sec. 2.1, Eq. 2.11-2.12, Prop. 2.6)
  decomposition  overlap extension (Def. 2.3), dof/ovdof (Def. 3.2), partition of unity (Def. 2.7)
  geneo          H_k-GenEO local eigenproblems (Def. of Eq. 5.12) and coarse space (Def. 5.1)
  schwarz        one- and two-level additive Schwarz (Eq. 2.22, 2.23)
  fgmres         right-preconditioned flexible GMRES (Euclidean inner product; the library's default solver)
  gmres_dk       left-preconditioned GMRES in the D_k inner product (the setting of Thm. 3.1, Eq. 2.24,
                 Prop. 2.6) and the theorem's quantities Lambda, tau, Theta, s, gamma
  solver         setup/solve pipeline mirroring the library's boundary

Parity status: every function is pinned by tests against closed forms,
invariants, brute force or an independent library route; the GMRES iteration
counts at the benchmark sizes are "parity unpinned" against the paper, which
prints no iteration counts.
"""
