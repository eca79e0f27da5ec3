"""Plain, slow, obviously-correct CPU FP64 oracle for the H1 mass/diffusion
operators on hexahedral Q_p meshes.

TEST INFRASTRUCTURE ONLY. Only the test-suite, the package entry point's
smoke check and the benchmark's CPU-baseline / reference arm may import this
package. It shares no code with the CUDA library (no kernels, headers, tables
or helpers); its only shared dependency is `fem_inputs`, which generates
seeded inputs and holds none of the method's arithmetic.

What it computes is the plain definition the partial-assembly method must
reproduce exactly up to rounding (Sec. 4.3-4.4: PA stores only D and applies
P, G, B on the fly, which is algebraically the same operator as the assembled
matrix with the same quadrature):

* 1D rules: Gauss-Lobatto-Legendre nodes (the nodal basis, Sec. 3.3) and
  Gauss-Legendre quadrature on [0,1] (`rules`);
* 1D Lagrange basis values/derivatives by the direct product formula
  (`lagrange`);
* the global DOF numbering: vertices, then edges, then faces, then element
  interiors (Sec. 3.4), computed from entity keys (`numbering`);
* dense element matrices by direct quadrature over all points:
  K_e = sum_q kappa_e w_q detJ (J^-T grad phi_i).(J^-T grad phi_j) and
  M_e = sum_q rho_e w_q detJ phi_i phi_j (Eqs. for A_ij and (M_E)_ij in
  Sec. 2 and Sec. 4.4) (`element`);
* global CSR assembly, SpMV and diagonal (`assemble`);
* essential-BC elimination, load vector, Jacobi-PCG and dense Cholesky
  (`solve`, Sec. 2 and Sec. 5.1);
* the compliance gradient dJ/dkappa_e = -u_e^T Khat_e u_e (`gradient`);
* the same definitions on quadrilaterals in 2D (`twod`);
* curved elements: the order-k nodal geometry of Sec. 3.1 in place of the
  trilinear map (`curved`);
* the convection operator (beta . grad u, v) (`convection`);
* linear elasticity on vector H1, lambda div div + 2 mu eps:eps
  (`elasticity`);
* p-multigrid: level hierarchy, nodal-interpolation transfers, coarse
  essential DOFs, Chebyshev-Jacobi smoothing, the V-cycle and flexible CG
  (`multigrid`; the paper names matrix-free p-multigrid, Sec. 5.2, without
  an algorithm: the module header states the reading);
* the assembled CSR product as a plain C loop, OpenMP over rows, for timing
  the CPU baseline on all host cores (`cspmv`, `spmv.c`; imported on
  demand, compiled by gcc).

Parity status: every function is pinned by `tests/test_oracle_*.py` against
closed forms, invariants or brute force, except the mixed-precision error,
which has no oracle of its own (parity unpinned beyond the FP64 outer
residual; the error against this FP64 oracle is reported per result).
"""

from . import (rules, lagrange, numbering, element, assemble, solve, gradient, twod, multigrid, curved,  # noqa: F401
               convection, elasticity)
