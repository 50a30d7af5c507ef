"""GB300-native unsteady discrete adjoint of the compressible Navier-Stokes equations
(arXiv 1511.06959): RK4 central finite-volume primal on periodic boxes, its exact
discrete adjoint with checkpoint recompute, the pressure-loss objective, the growth
matrix sigma_1 and the added adjoint viscosity, all as sm_103a CUDA kernels behind a
C ABI.  Importing the package loads nothing; ``paper_1511_06959_gb300.api`` loads the
CUDA library and fails loudly if it is missing."""
