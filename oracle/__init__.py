"""Plain FP64 CPU oracle for the (X)MS-CASPT2 amplitude, lambda and density path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline leg of bench.py may import this package.  The product library never
calls it and shares no code with it; the two meet only through the seeded
inputs of the `synth` package.

  o1_determinant  brute force in the full determinant space (tiny spaces):
                  explicit excitation operators, explicit overlap / zeroth-order
                  Hamiltonian matrices, explicit expectation values.
  mp2_closed_form textbook closed-shell MP2 (nact = 0 special case), used as a pin.
  o2_rdm, o2_classes, wick
                  RDM / orbital-tensor form for sizes the brute force cannot reach
                  (class H pair form; classes A-G from a spin-free normal-ordering
                  engine), pinned against o1_determinant.
  o2_offdiag      off-diagonal blocks of the density d-bar(2) (class-to-class couplings
                  through E_xy), pinned against o1_determinant.
  o1_orbderiv     orbital derivative Y of the Lagrangian from o1_determinant's densities.
  o1_cideriv      CI derivative, XMS multipliers w_MN and the XMS terms Y', y~'.
  o1_iterative    iterative solve of the coupled amplitude equations (subspace residual
                  minimisation), with warm starts.
  (each pinned against finite differences or the direct solve of o1_determinant)
"""
