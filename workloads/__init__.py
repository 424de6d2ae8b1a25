"""Seeded synthetic inputs for finite-element assembly.

This module produces the two inputs that the assembly problem of Sky et al.
(arXiv 2012.00585, §2.1 "A generic element") is stated in terms of:

* ``elem_dofs``  -- the element-to-DOF connectivity (``element_dofs_array``),
  an ``int32 [n_e, n_loc]`` row-major array, local order per element;
* ``K``          -- the dense element matrices, ``float64 [n_e, n_loc, n_loc]``
  row-major per element.

It holds no assembly arithmetic: no sparsity pattern, no scatter, no search.
Both the CPU oracle (``oracle/``) and the CUDA path consume what it makes,
and neither is imported here.

The paper measured on Gmsh square meshes that are not available; the
structured and Kuhn-split meshes below stand in for them (same element
families, same DOF-per-node interleaving ``dof = d*node + comp``).
"""

from .meshes import (  # noqa: F401
    quad_q1_grid,
    quad_qp_grid,
    hex_q1_grid,
    tet_p2_kuhn,
    batched_mesh_sizes,
    paper_sweep_points,
)
from .elements import (  # noqa: F401
    laplace_q1_quad,
    laplace_q1_hex,
    elasticity_q1_hex,
    ones_matrices,
    broadcast_matrices,
    random_spd_matrices,
    random_matrices,
    scaled_matrices,
)
