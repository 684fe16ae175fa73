"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds geometry and excitation generators only: triangle meshes
of the paper's benchmark scatterers (Section 2.1: a square plate in the x-y
plane and a sphere, both centred at the origin and meshed at about lambda/9),
plane-wave incidence directions and polarisations, and seeded random vectors.
It contains none of the method's arithmetic (no basis functions, quadrature,
Green's function, projection or solver), so both the CPU oracle and the CUDA
path may consume its output without sharing any of the method.
"""

from .meshes import plate_mesh, rect_plate_mesh, icosphere_mesh, icosphere_frequency, mesh_mean_edge
from .incidence import (
    planewave_minus_z_xpol,
    random_incidence,
    sphere_four_directions,
    random_complex,
)

__all__ = [
    "plate_mesh",
    "rect_plate_mesh",
    "icosphere_mesh",
    "icosphere_frequency",
    "mesh_mean_edge",
    "planewave_minus_z_xpol",
    "random_incidence",
    "sphere_four_directions",
    "random_complex",
]
