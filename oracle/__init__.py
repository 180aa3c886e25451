"""Plain, slow, obviously correct CPU oracle for the FMM-BEM hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, bench.py's cpu_baseline / reference
leg and __graft_entry__.smoke() may import, call or run anything here; the
product (paper_2103_01048_gb300) never does, and shares no code with it.

Modules
  kernels        FP64 direct sums of the Laplace/Yukawa single- and
                 double-layer kernels (Eq. nbody_sum with the kernels of
                 Eq. single_double and Eq. adj_hyp), via the C file oracle.c.
  tree           adaptive octree and U/V/W/X interaction lists (Sec. "Fast
                 multipole method"), plain recursive definition.
  bem            P0 Galerkin discretisation of the direct formulation
                 (Eq. direct), dense assembly and LU solve, reaction
                 potential (Eq. phi_reac) and polar solvation energy
                 (Eq. energy).
  closed_forms   Born ion and Kirkwood sphere energies (Sec. "Mesh
                 refinement study using an analytical solution").

Parity status: every function here is pinned by a `-m "not gpu"` test in
tests/test_oracle_*.py against closed forms, brute force or printed values.
"""
from ._lib import lib, build_oracle  # noqa: F401
