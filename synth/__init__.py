"""Seeded synthetic inputs: tetrahedral meshes, material tables, initial
magnetisations and field sweeps.

This package only *generates inputs*.  It contains none of the arithmetic of
the minimisation method (no finite-element assembly, no energies, no solvers),
so both the CUDA path and the CPU oracle may use it without sharing any of the
method's code.
"""
from .mesh import Mesh, kuhn_lattice, cube_in_box, jitter_nodes, voronoi_regions, grain_patches
from .workloads import (Workload, soft_cube, hard_cube, polycrystal_cube,
                        small_cube, random_unit_vectors, cone_axes, platelet,
                        platelet_batch, graded_cube_in_box, large_polycrystal, sp3_cube,
                        sphere_in_box)

__all__ = ["Mesh", "kuhn_lattice", "cube_in_box", "jitter_nodes",
           "voronoi_regions", "grain_patches", "Workload", "soft_cube", "hard_cube",
           "polycrystal_cube", "small_cube", "random_unit_vectors",
           "cone_axes", "platelet", "platelet_batch",
           "graded_cube_in_box", "large_polycrystal", "sp3_cube", "sphere_in_box"]
