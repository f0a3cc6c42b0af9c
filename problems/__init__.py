"""Seeded synthetic inputs for the RAS solver and its oracle.

This package builds the linear systems Ax = b that both the CUDA path and the
CPU oracle consume: the 2D/3D Poisson stencils of the experimental section
(Sec. 4.1: 5-point stencil S = {-1,-1,4,-1,-1}), a variable-coefficient 2D
diffusion operator with a log-normal random coefficient, a nonsymmetric
upwind convection-diffusion operator, uniform random
right-hand sides and the discrete eigenvector right-hand side.

It holds none of the Schwarz method's arithmetic (no partitioning, overlap,
local solves or iteration); it only produces matrices and vectors.
"""
from .generators import (  # noqa: F401
    splitmix64,
    uniform01,
    normals,
    poisson2d,
    poisson3d,
    diffusion2d,
    convdiff2d,
    rhs_eigen_convdiff2d,
    grf_coefficient,
    rhs_uniform,
    rhs_eigen2d,
    rhs_eigen3d,
    CSR,
)
