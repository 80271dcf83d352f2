"""Seeded synthetic inputs for the SBFEM full-waveform-inversion workloads.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle.  It only *generates inputs*: mesh coordinates and connectivity, density
fields on a fine Cartesian grid, source wavelets, source/receiver node choices
and the time-step size.  It holds none of the method's arithmetic (no shape
functions, no coefficient matrices, no condensation, no time stepping).

The workloads stand in for the paper's flawed-specimen experiments
(Section 4: a plate with a hole and a plate with a weak inclusion, sources on the
top surface, receivers along the edges), whose FEM-generated data and Voronoi
meshes are not available.  They use square S-elements (structured or quadtree
meshes, and the paper's centroidal Voronoi polygons), a void/flaw density contrast,
and Ricker or sine-burst sources.
"""

from .mesh import (StructuredMesh, structured_mesh, boundary_nodes, nearest_node, QuadtreeMesh, quadtree_mesh,
                   min_spacing, PolygonMesh, voronoi_mesh)
from .fields import flawed_density_circle, flawed_density_ellipses
from .wavelet import ricker, sine_burst
from .configs import (Workload, tiny_workload, size_workload, diff_workload, paper_workload, batching_workload,
                      solid_workload, workload_by_name)

__all__ = [
    "StructuredMesh", "structured_mesh", "boundary_nodes", "nearest_node", "QuadtreeMesh", "quadtree_mesh",
    "min_spacing", "PolygonMesh", "voronoi_mesh", "batching_workload",
    "flawed_density_circle", "flawed_density_ellipses", "ricker", "sine_burst",
    "Workload", "tiny_workload", "size_workload", "diff_workload", "paper_workload", "solid_workload",
    "workload_by_name",
]
