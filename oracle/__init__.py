"""FP64 CPU oracle for the generalized Yee method (GYM) leapfrog step.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import anything from here.  The
product path (the C-ABI library and its Python binding) never imports, links
or calls this package, and this package never imports the product.

The oracle is a plain, slow, obviously-correct restatement of the paper:
  mesh.py      structured PEC cube split into Kuhn tetrahedra, DoF numbering
  basis.py     order-k trimmed (P_k^-) 1-/2-form bases in barycentric form,
               tetrahedron quadrature
  fem.py       mass matrices M1(eps), M2(mu) (Sec. 2), integer G, C, D of the
               discrete de Rham complex (Eq. discreteDeRham), load vectors,
               canonical edge interpolation
  spai.py      column-wise SPAI on a sparsity pattern (Eq. NormalEqSolve)
               followed by symmetrisation (Sec. 5)
  spai_op.py   operator-probed SPAI: the symmetric Sylvester system of
               Eq. SPAIOPSylvester solved by diagonally preconditioned CG (Sec. 5.1)
  adjoint.py   reverse sweep of the leapfrog and the eps-derivative of the column
               SPAI: gradient of a probe-region field energy (order 1)
  gym.py       shear maps / Strang splitting (Eqs. shearMaps, strangSplit),
               the (b, e) leapfrog (Eq. preYeeFEECEqns, Eq. YeeLeapfrog),
               energies, CFL bound (Prop. stability), dipole source
  cubical2d.py 2-D periodic cubical Whitney GYM used only to pin the SPAI and
               dispersion numbers printed in Table dispersionTable

Parity status per function is stated in each module header.
"""
