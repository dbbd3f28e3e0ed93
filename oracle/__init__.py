"""Plain FP64 CPU oracle for the ROM-accelerated minimum-compliance SIMP method.

TEST INFRASTRUCTURE ONLY. This package restates, slowly and obviously, what the CUDA
library computes, so that the library can be checked against it. Only the tests, the
smoke check of the package entry point and the CPU-baseline leg of the benchmark may
import it. The product path never calls it, links it or falls back to it.

It shares no code with the CUDA path: its element matrices come from its own quadrature,
its operator is an assembled scipy.sparse matrix, its solves are direct (SuperLU) or its
own CG, and its reduced model uses numpy's Householder QR and scipy's Cholesky. The only
shared module is the seeded input generator (workloads), which holds no method arithmetic.

Modules:
  element  -- unit-density Q4 / H8 element stiffness (Section 2.1, Eq. linelast-res1)
  fem      -- assembly, Dirichlet elimination, solve, compliance, gradient (Sections 2.1-2.4)
  hatfilter-- linear (cone) density filter and its adjoint (the benchmark's filter)
  rom      -- Galerkin ROM, residual, error bounds (Sections 3.1-3.3)

Parity status: every function here is pinned by tests against closed forms, invariants,
exact symbolic integration, finite differences or brute force (see tests/test_oracle_*.py),
except where a function's docstring says "parity unpinned".
"""
