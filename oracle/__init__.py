"""CPU oracle for algebraic hPLMM (Khan & Mehmani, "High-order Multiscale
Preconditioner for Elasticity of Arbitrary Structures").

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
the paper's definitions, written to check the CUDA library against.  Only the
test-suite, the package-level smoke check and the benchmark's CPU-baseline leg
may import it; the library itself never does, and the two share no code other
than the seeded input generators in `synth`.

Modules, in the paper's order:
  fem           Section 2, Eqs. stiff_iso and ls_all: Q1 hexahedra on voxels, loads, Dirichlet elimination
  decomposition Section 3.1-3.2 and Eq. permute: Cartesian grain grids, contact interfaces, permutation W
  mortar        Section 3.3, Eqs. node_init and gauss: mortar-node placement, Gaussian mortars, Q^o
  coarse        Section 4.2, Eqs. mg_struct, WQP, bc_matrix, col_cg, col_pk: prolongation and coarse solve
  smoother      Section 4.3, Eqs. local_smoother_CG and Mg_Mz: contact-grain additive-Schwarz smoother
  precond       Section 4.1, Eqs. multi_precond and local_smoother: the multiplicative two-level M
  ilu           Sections 4.1 and 5: the ILU(0) base smoother of the paper's smoother comparison
  spectral      Section 3.1: spectral k-way partition of a gray-scale image into grain grids
  gmres         Section 5: right-preconditioned restarted GMRES
  accuracy      Eq. err_metric: first-pass L2 errors of displacement and maximum shear stress
  warmstart     learned warm start of the local basis solves (3-D convolutional network, Adam) and the
                block-Jacobi preconditioned CG basis solver it feeds (an optional iterative path beside the
                paper's exact local solves of Eqs. col_pk and col_cg)

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, invariants or brute force; see the pin list in each module.
"""
