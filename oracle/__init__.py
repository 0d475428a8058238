"""CPU oracle for the thermoelastic SA-AMG-PCG path (TEST INFRASTRUCTURE ONLY).

This package is a plain, slow, FP64 restatement of what the paper's method
computes, written to check the CUDA library.  Only the test-suite, the smoke
check and the CPU-baseline leg of the benchmark may import it; the product
path never does, and it shares no code with the CUDA sources.

* ``oracle.fem``      -- element integrals (exact, via barycentric monomial
  integration), assembly, Dirichlet elimination, rigid-body modes.
* ``oracle.linsolve`` -- dense Cholesky, sparse direct and Jacobi-PCG solves.
* ``oracle.amg``      -- smoothed-aggregation AMG pieces and the AMG-PCG solve.
* ``oracle.thermal``  -- the heat equation of the thermal half of the model:
  theta-method residual and Newton Jacobian with Robin faces, Newton, and
  the adaptive time step.

Parity status per function is stated in each module header.
"""
