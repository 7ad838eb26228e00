"""Seeded synthetic workloads for the shifted-solve path of projection MOR.

This package only *generates inputs* (sparse matrices, input/output vectors,
initial shifts).  It contains none of the arithmetic of the method itself
(no shifted operator, no preconditioner, no Krylov, no projection), so that
the CPU oracle and the CUDA path can both consume it without sharing any
method code.

The paper's own test models (disk brakes from Grabner et al.) are not
available; the generators here stand in for them with stencil systems of the
same size and sparsity class:

  * laplace2d_siso          2D 5-point Laplacian, n = 10,000, E = I, SISO
  * convdiff3d_siso         3D 7-point upwind convection-diffusion, n = 1,000,000,
                            E diagonal
  * uneven_laplace2d_batch  256 uneven 2D Laplacian-plus-diagonal systems,
                            n_s in [2000, 60000]
  * stencil27_second_order  3D 27-point SPD stencil, second order, Rayleigh
                            damping, n = 1,197,900
  * convdiff3d_mimo         3D 7-point convection-diffusion, n = 8,000,000,
                            MIMO m = q = 8
"""
from .generators import (  # noqa: F401
    Workload,
    SecondOrderWorkload,
    laplacian_2d,
    convection_diffusion_3d,
    stencil27_3d,
    laplace2d_siso,
    convdiff3d_siso,
    uneven_laplace2d_batch,
    stencil27_second_order,
    convdiff3d_mimo,
    csr_arrays,
    random_sparse_system,
)
