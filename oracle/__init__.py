"""FP64 CPU oracle for inner-outer Krylov recycling (arXiv 1602.00138).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
bench's CPU-baseline / reference legs may import anything in this package.
The product path (the CUDA library and its Python binding) never imports it
and shares no code with it: the oracle assembles the full finite-difference
system with explicit Robin boundary unknowns and forms the Schur complement
numerically, while the CUDA path applies closed-form stencil coefficients.

Contents (each function cites the passage of the paper it restates):
  operator  -- full system (Sec. 2.1, Sec. 3 eq. block1), Schur complement
               A~ = F - D2 G^-1 D1 and effective sources B~, C~ (Sec. 3.1).
  solvers   -- dense / sparse direct solves, plain CG, deflated CG
               (Saad, Yeung, Erhel & Guyomarc'h 2000).
  eigen     -- smallest eigenvectors of A~_0 (Sec. 4.2.2).
  basis     -- Algorithm 2 (Sec. 4.3) in sequential and wave order, with the
               ordered rank-revealing append; the per-RHS recycling of the
               Sec. 6.3 comparison (Table 2).
  minres    -- the paper's minimum-residual check (eq. initialz) and
               recycled MINRES on the projected operator (Sec. 4.1, eqs.
               eq01, SmallMin).
  rom       -- reduced transfer function and Jacobian (Sec. 3.3-3.4, eqs.
               newreduced, newjac) and the full-order plain definitions.
  cnn       -- the learned augmentation of the private recycle space (not
               in the paper): coarse 3D CNN forward pass, features, loss.

All arithmetic is float64.  Parity status of each function is recorded in
its docstring; every function here is pinned by a -m "not gpu" test against
an independent fact (closed forms, dense direct solves, finite differences,
reciprocity, invariants of the algorithm).
"""
