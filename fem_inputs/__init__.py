"""Seeded synthetic inputs for the PA finite-element path.

This package is shared by the tests, the benchmark and the CPU oracle. It
holds only input generation: a counter-based random generator, structured-
topology hexahedral meshes passed on as unstructured (coords, hex) arrays,
per-element coefficients and input vectors. It contains none of the method's
arithmetic (no quadrature, no basis functions, no Jacobians).

Workload recipes (the shapes of the paper's workloads, Sec. 5.3 and the
partial-assembly discussion of Sec. 4.4):

* unit cube [0,1]^3 cut into N^3 hexahedra of size h = 1/N;
* every vertex coordinate moved by an independent U[-a*h, a*h] draw; a
  vertex on the boundary moves only tangentially (corners stay, edge vertices
  slide along their edge, face vertices stay in their face), so the domain
  stays exactly the unit cube;
* optional shuffling of vertex and element numbering and a random proper
  rotation of each element's local vertex order (exercises shared-entity
  orientation handling);
* curved meshes: per-element nodal coordinates at an equispaced lattice,
  the multilinear vertex map followed by a smooth bulge that fixes the
  domain boundary (the library and the oracle read them as the element's
  order-k nodal geometry);
* per-element coefficient kappa_e with log(kappa_e) ~ N(0, 1);
* input vectors x ~ U[-1, 1].
"""

from .rng import splitmix64, uniform01, uniform, normal, permutation
from .mesh import hex_lattice, CUBE_ROTATIONS, lattice_dofs, submesh, quad_lattice, curved_nodes
from .fields import lognormal, x_uniform, rho_uniform

__all__ = [
    "splitmix64", "uniform01", "uniform", "normal", "permutation",
    "hex_lattice", "CUBE_ROTATIONS", "lattice_dofs", "submesh", "quad_lattice", "curved_nodes",
    "lognormal", "x_uniform", "rho_uniform",
]
