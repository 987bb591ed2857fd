"""CPU FP64 oracle for the multiresolution SIMP elasticity solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` use it.  It shares no
code with the CUDA path (no kernels, tables, constants or helpers).

It computes, plainly and slowly, what the GPU path computes:
  fem      -- element shape functions, D, B and the subcell stiffness table
              K^(e_i) = int_{subcell i} B^T D B (Section 3.3, Eq. matrixK_mr)
  mesh     -- node lattice, element DOF lists, density-cell <-> subcell map
  filt     -- the Gaussian density filter / design projection matrix H
              (Section 2.2 Eq. filter_weights, Section 3.2 Eq. projdsgn)
  fe       -- SIMP weights, sparse assembly of K(rho) (Eqs. matrixK and
              matrixK_mr), Dirichlet elimination, direct / CG solve,
              compliance f^T u, subcell energies and the gradient
              (Section 3.4)
  mg       -- the geometric multigrid cycle of Algorithm 1 (Section 2.3)
              with Jacobi smoothing and a dense Cholesky coarse solve, and
              preconditioned CG (Section 7.2)

Every function is FP64.  "parity unpinned" is stated where a function has no
pin other than itself (see the individual docstrings); all others are pinned
by tests in tests/test_oracle_*.py.
"""
