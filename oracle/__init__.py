"""FP64 CPU oracle for MGAR / MGCG heat-transfer topology optimisation.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this package.  The CUDA library
never calls it, and it shares no code with the CUDA library: the two only
draw their inputs from the same seeded generators.

Everything here is plain numpy / scipy.sparse in float64, written to be read
against the paper (Yin, Wang, Guo, Li, "An efficient topology optimization
based on multigrid assisted reanalysis for heat transfer problem",
arXiv 2210.00947):

  fem.py        Eq. 3-4   Galerkin FE conductivity matrix with SIMP
  multigrid.py  Table 1   transfer operators, Galerkin coarse operators,
                          damped Jacobi, recursive V-cycle
  solvers.py    Eq. 12-21, 28 and Section 3.2: MGCG, MGAR, exact solve
  design.py     Eq. 5-11  density filter, compliance, sensitivities, and
                the optimality-criteria update (not in the paper)
  loop.py       Section 3.1 (Figure 5): the MGAR-based optimisation loop

Readings taken where the paper is silent are stated where they are used.
Parity status: every function is pinned by the CPU tests except where its
docstring says "parity unpinned".
"""
