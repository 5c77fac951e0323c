"""Plain, slow, FP64 CPU oracle of the IMEX multi-rate SDC heat simulation.

TEST INFRASTRUCTURE ONLY. Nothing in the library or its product path may
import, call, link or run anything in this package; it exists so that tests,
the smoke check and the CPU-baseline leg of the benchmark can check the CUDA
path against an independent, obviously correct restatement of the paper.

Modules
-------
weights   quadrature nodes and the four MRSDC weight tables (Sec. 3, the
          weight definitions after Eq. (embedded_quad) and Table 1), in exact
          rationals or 60-digit arithmetic.
fem       trilinear finite elements: lumped mass, stiffness, Robin terms
          (Sec. 2, Eqs. femContFix/femContMov and the matrix definitions).
contact   the explicit coupling term f^E(T, t) on the moving contact patch,
          by brute-force intersection of every stand/stock face pair (Sec. 2,
          the definitions of b_X(t), M_B and C_B).
linsolve  Jacobi-preconditioned CG and dense Cholesky for (M + dtau K) x = b.
mrsdc     Algorithm 1 (predictor) and Algorithm 2 (sweep) taken literally,
          with full vectors at every embedded node, plus the residual of
          Eq. (residual).
machine   the coupled stand/stock problem object built from `synth` inputs.

Parity status of each function is stated in its module docstring; every
function here is pinned by a test under tests/ against a value fixed by the
paper or by mathematics, not against the CUDA path.
"""
