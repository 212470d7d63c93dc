"""CPU FP64 oracle for the Recursive Schur Decomposition preconditioner.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the bench's CPU
baseline leg may import, call or execute anything in this package; the product
library never does, and this package imports nothing from the product.

Modules and what each follows:
  fem        trilinear FEM on a structured cube grid (Sec. 4's discretisation in 3-D)
  partition  octree decomposition, ownership, interface sets (Sec. 2; Eq. 3.1)
  rsd_exact  exact recursive Schur complements and substitution (Eqs. 3.2-3.3, Sec. 3.2)
  rsd_paper  Algorithm 2 with the V-hat truncation and Algorithm 1 (Sec. 3.2-3.3)
  krylov     PCG and flexible GMRES (the outer solver of Sec. 3)
  problem    convenience: a synthetic workload -> matrix, load, owner map, tree
  adjoint    adjoint solve and per-element coefficient gradient of u = K(kappa)^-1 b

Functions with no independent pin are marked "parity unpinned" in their docstring;
currently there are none.
"""
