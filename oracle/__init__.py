"""Plain FP64 CPU oracle for the Poisson-lognormal MAP solve.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
definition that the CUDA library is checked against.  Only the test suite,
the smoke check and the CPU-baseline leg of the benchmark may import it; the
library itself never does, and the oracle never imports the library.  The two
share no code: the oracle has its own DFT (a separable matrix DFT, pinned to a
brute-force 3D DFT), its own prior spectrum, its own Lambert W and its own
Newton-Krylov iteration.

Modules
  dft       -- discrete Fourier transform by definition (Sec. 2.2: the prior
               covariance is a convolution, diagonal in Fourier space).
  lambertw  -- principal-branch Lambert W, for the diagonal-prior closed form.
  plc       -- prior spectrum, objective, gradient, Hessian-vector product,
               preconditioned CG, Newton-Krylov MAP and its implicit adjoint
               (Sec. 2.1, 2.3, 3.1, 3.1.2).

Every function is pinned by a test against something other than itself
(closed forms, brute force, finite differences, invariants); see tests/.
"""
