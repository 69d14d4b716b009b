"""Plain FP64 CPU oracle for the multigrid V-cycle of Takacs, "Fast multigrid
solvers for conforming and non-conforming multi-patch Isogeometric Analysis"
(arXiv:1902.01818).

TEST INFRASTRUCTURE ONLY. Nothing here is part of the product: only the test
suite, the smoke check and the CPU-baseline leg of the benchmark may import it.
It shares no code with the CUDA library and imports nothing from it.

Everything is written for clarity, not speed: numpy/scipy arrays in float64,
scipy.sparse for assembled matrices, LAPACK (through scipy) for dense
factorisations.  Each function cites the paper's section or equation it
follows.  Where the paper is silent the reading taken is stated in the
docstring.

Modules
  bspline     -- knot vectors, Cox-de Boor basis, Gauss-Legendre rules (Sec. 2)
  geometry    -- tensor-product B-spline geometry maps G_k (Sec. 2, Eq. omega:2)
  discretize  -- DoF numbering, Galerkin and SIPG assembly (Sec. 2, Sec. 3)
  hierarchy   -- grid levels, knot-insertion prolongation, Galerkin coarse
                 operators (Sec. 3 Eq. a:galerkin, Sec. 4)
  pieces      -- piece decomposition of the DoFs (Sec. 5)
  smoothers   -- subspace-corrected mass smoother, Gauss-Seidel (Sec. 4-6)
  mg          -- V-cycle (Algorithms 1 and 2), PCG, error propagation (Sec. 4)

Parity status: every function is pinned by a CPU test against a closed form,
an invariant or brute force, except the iteration counts of the paper's own
tables, which cannot be reproduced (their geometry files are not published):
that comparison is "parity unpinned".
"""
