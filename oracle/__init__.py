"""CPU FP64 oracle for periodic voxel homogenization — TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously-correct reference that the CUDA library is
checked against. Only the test suite, the smoke check and the benchmark's CPU-baseline
leg may import it; the product path never calls it, and it shares no code with the CUDA
library (the two only see the same voxel arrays, produced by the seeded generators).

Modules:
  fe        element matrices (hex8 elasticity and heat) and affine macro modes (App. F)
  grid      sparse hierarchy: active elements/nodes, octant masks, coarsening, transfer
            stencils (Sec. 4.1 "Solver-Aligned Hierarchy Construction", App. E)
  solve     global assembly, conjugate-gradient solve, dense brute force, residual and
            the energy-averaged homogenized tensor (Sec. 3.1, Sec. 5 metrics, App. F)
  galerkin  global prolongation matrix and Galerkin coarse operators (Sec. 3.2, Sec. 4.6)
  unet      the learned initializer's sparse convolutional U-Net, its loss, autograd
            gradient and AdamW step (Sec. 4.2-4.3, Alg. 2)

Parity pins: every function here is checked in tests/ against closed forms, invariants
or brute force (see the test files); no function is "parity unpinned".
"""
