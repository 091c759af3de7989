"""CPU FP64 oracle for CNN-preconditioned FGMRES on the 2D Helmholtz equation.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
It shares no code with the CUDA library (no kernels, headers, helpers,
tables or constants); the only common module is the seeded input generator
`paper_2607_16906_b300.synth`, which draws numbers and holds none of the
method's arithmetic.

Modules:
  helmholtz  PML profiles (eq. 2), the complex-symmetric 5-point operator as a
             scipy CSR matrix and as a matrix-free stencil, its adjoint, the
             sparse direct solve, the free-space Green's function (eq. 1).
  unet       the 4-level U-Net (Sec. 3.1, read as 16/32/64/128 channels,
             3x3 convs, ReLU) forward and backward in plain numpy FP64, with
             an optional BF16 emulation of the conv inputs.
  fgmres     flexible GMRES (Alg. 1, eq. 4) with CGS2 or MGS, complex Givens,
             restarts and an FP64 iterative-refinement driver.
  train      the physics-informed loss (eqs. 8-9), its gradient, AdamW.

Every function is pinned by a `-m "not gpu"` test against something other
than itself (closed forms, library routines, brute force, invariants).
Pinning status per function is listed in each module's header.
"""
